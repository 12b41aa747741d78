// tsvd_api.cu -- the C ABI of libtsvd (include/tsvd.h): argument checks, device workspaces,
// host/device staging and the order of kernel launches of the t-SVT and of the two ADMM
// solvers.  All arithmetic runs in the kernels of tube_pass.cu and slice_svt.cu; this file
// only computes the scalar penalty schedule rho_k (Sec. 4 / Sec. 5) on the host.
#include "tsvd.h"
#include "tsvd_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

using namespace tsvd;

struct tsvd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  tsvd_opts opts{};
  std::string err;
  char* ws = nullptr;        // device workspace
  size_t ws_cap = 0;
  std::vector<float2> twid_host;   // kept alive while copies may be in flight
  std::vector<int> slices_host;
  std::vector<unsigned char> isreal_host;
  std::vector<SliceStat> stat_host;
  // launch accounting of the current call
  int64_t launches = 0;
  int64_t slice_launches = 0;
  // opts.timing: event pairs around launches; kind 0 = slice SVT, 1 = tube pass
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kind;
  size_t events_used = 0;
  // autotuned slice-SVT plans, keyed by (n1, n2, slices per launch, V form)
  std::map<std::array<int, 4>, SliceKnobs> tuned;
  bool cache_loaded = false;
  // CUDA graphs of whole solver launch sequences, keyed by everything the launches depend on
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0, slice_launches = 0;
    size_t events_used = 0;
  };
  std::map<std::vector<int64_t>, Graph> graphs;
  cudaStream_t cap_stream = nullptr;   // private stream used only for capture
  cudaStream_t cur = nullptr;          // stream the launch helpers enqueue on
  bool capturing = false;              // a launch sequence is being captured
  // batched solves: parallel stream branches and their fork / join events
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  // plain form: the current solve runs the V form (warm start), for the plan lookups
  bool vform_now = false;
  // persistent batched solves: tuned (cluster size, single-CTA threshold) per batch shape, and
  // the host copy of the device table (alive while its copy may be in flight)
  std::map<std::vector<int64_t>, std::array<int, 2>> batch_tuned;
  std::vector<unsigned char> batch_table;
  // tsvd_factor: converged vectors, rotations, Fourier-domain factors and output staging
  char* fbuf = nullptr;
  size_t fbuf_cap = 0;
  // mixed form: per-iteration sketch statistics copied to pinned host memory (a ring read
  // two iterations late, so the host never waits for the iteration it just enqueued)
  static constexpr int kRing = 4;
  RsvtStat* rs_host = nullptr;
  cudaEvent_t rs_ev[kRing] = {};
  int rs_k_last = 0;
  int64_t rs_saturated = 0, rs_drops = 0;
  double rs_gemm_gflop = 0, rs_svd_gflop = 0;
  // opts.timing: stage events of every randomized SVT of the current call
  std::vector<std::array<cudaEvent_t, 7>> rs_stage;
  size_t rs_stage_used = 0;
};

namespace {

constexpr size_t kAlign = 256;

// ---- host-side fault injection: TSVD_FAULT="alloc:N" makes the N-th device allocation of the
// library in this process (counting from 1) fail as if the device were out of memory, so the
// TSVD_ENOMEM paths can be exercised without exhausting a GPU.  Read at the first allocation
// (or by tsvd_fault_injection_reset).
std::atomic<long long> g_fault_alloc_at{-1};   // -1: not read yet; 0: off
std::atomic<long long> g_alloc_count{0};

long long parse_fault_spec(const char* spec) {
  if (!spec) return 0;
  const char* pre = "alloc:";
  if (std::strncmp(spec, pre, std::strlen(pre)) != 0) return 0;
  char* end = nullptr;
  const long long n = std::strtoll(spec + std::strlen(pre), &end, 10);
  return (end && *end == '\0' && n > 0) ? n : 0;
}

// cudaMalloc, unless the fault injector says this allocation fails.
cudaError_t device_alloc(void** ptr, size_t bytes) {
  long long at = g_fault_alloc_at.load();
  if (at < 0) {
    at = parse_fault_spec(std::getenv("TSVD_FAULT"));
    long long expect = -1;
    g_fault_alloc_at.compare_exchange_strong(expect, at);
    at = g_fault_alloc_at.load();
  }
  const long long n = ++g_alloc_count;
  if (at > 0 && n == at) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

// A named range of the library's host-side work for profilers (NVTX; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

tsvd_status fail(tsvd_ctx* c, tsvd_status st, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

#define TSVD_CUDA(ctx, expr)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaGetLastError(); /* do not leave a non-sticky error for a later launch check */  \
      return fail((ctx), TSVD_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
    }                                                                                     \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// 0 = device-accessible on `dev`, 1 = host memory, -1 = device memory of another device.
int pointer_kind(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? 0 : -1;
  if (at.type == cudaMemoryTypeManaged) return 0;
  return 1;
}

// The mixed form: randomized slice SVT (every precision but plain FP32 Jacobi).
bool mixed_precision(const tsvd_ctx* c) { return c->opts.precision != TSVD_PRECISION_FP32; }

// Problem geometry shared by every entry point.
struct Problem {
  int order = 0;
  int64_t n1 = 0, n2 = 0, n3 = 0, n4 = 1;
  int64_t N = 0;       // entries
  int64_t nslices = 0; // Fourier slices of the full spectrum (n3 or n3*n4)
  TubeGeom g{};
};

// Validates dims and fills the geometry.  need_svd: the call runs slice SVDs (their size
// limits apply); the t-product runs none.
tsvd_status make_problem(tsvd_ctx* c, int order, const int64_t* dims, Problem& p,
                         bool need_svd = true) {
  if (!dims) return fail(c, TSVD_EINVAL, "dims is NULL");
  if (order < 3 || order > 6) return fail(c, TSVD_EINVAL, "order must be 3 to 6 (got %d)", order);
  for (int d = 0; d < order; ++d)
    if (dims[d] < 1) return fail(c, TSVD_EINVAL, "dims[%d] = %lld < 1", d, (long long)dims[d]);
  p.order = order;
  p.n1 = dims[0];
  p.n2 = dims[1];
  for (int d = 2; d < order; ++d)
    if (dims[d] > (1 << 20)) return fail(c, TSVD_EUNSUPPORTED, "extent too large");
  if (p.n1 > (1 << 30) || p.n2 > (1 << 30)) return fail(c, TSVD_EUNSUPPORTED, "extent too large");
  // modes 3..N-1 take the full DFT (their flattened index kf, mode 3 fastest), mode N the
  // half-spectrum DFT
  int64_t nf = 1;
  for (int d = 2; d < order - 1; ++d) nf *= dims[d];
  if (order >= 5 && nf > 64)
    return fail(c, TSVD_EUNSUPPORTED, "modes 3..%d hold %lld entries per tube section (at most 64)",
                order - 1, (long long)nf);
  if (nf > (1 << 20)) return fail(c, TSVD_EUNSUPPORTED, "extent too large");
  p.n3 = order == 3 ? dims[2] : nf;
  p.n4 = order == 3 ? 1 : dims[order - 1];
  p.nslices = nf * dims[order - 1];
  if (p.n1 * p.n2 > (INT64_MAX / 16) / p.nslices)
    return fail(c, TSVD_EUNSUPPORTED, "tensor too large");
  p.N = p.n1 * p.n2 * p.nslices;
  p.g.N12 = p.n1 * p.n2;
  p.g.nf = (int)nf;
  p.g.nh = (int)dims[order - 1];
  p.g.hh = p.g.nh / 2 + 1;
  p.g.nstore = p.g.nf * p.g.hh;
  p.g.nfm = order - 3;
  for (int d = 0; d < p.g.nfm; ++d) p.g.fdim[d] = (int)dims[2 + d];
  if (!tube_pass_supported(p.g))
    return fail(c, TSVD_EUNSUPPORTED, "tube of %lld entries exceeds the tube-pass limit",
                (long long)p.nslices);
  if (!need_svd) return TSVD_OK;
  if (mixed_precision(c)) {
    // the randomized SVT only runs Jacobi on the projected nw x k matrices
    const int nw = (int)std::min(p.n1, p.n2);
    if (!jacobi_svt_supported(nw, std::min(nw, rsvt_max_k())))
      return fail(c, TSVD_EUNSUPPORTED, "slices with min(n1, n2) = %d are not supported", nw);
    return TSVD_OK;
  }
  if (!jacobi_svt_supported((int)p.n1, (int)p.n2))
    return fail(c, TSVD_EUNSUPPORTED,
                "a %lld x %lld complex slice does not fit one SM's shared memory",
                (long long)p.n1, (long long)p.n2);
  return TSVD_OK;
}

// float2 entries of the twiddle region: the half-mode and full-mode tables, and for more than
// one full mode the DFT matrix and the partner table (ints in float2 slots).
size_t twid_count(const TubeGeom& g) {
  size_t n = (size_t)g.nh + g.nf;
  if (g.nfm >= 2) n += (size_t)g.nf * g.nf + ((size_t)g.nf + 1) / 2;
  return n;
}

// The twiddle region of a tube geometry, in FP64 and rounded once: (cos, sin)(2 pi m / n) for
// the half mode (n = nh) and the full mode (n = nf), exact at the quarter points; for more
// than one full mode also the nf x nf matrix of their multi-dimensional DFT (the product of
// the modes' twiddles) and the conjugate partner of every full index.
void fill_twiddles(const TubeGeom& g, std::vector<float2>& out) {
  auto table = [](int n, float2* dst) {
    for (int m = 0; m < n; ++m) dst[m] = twiddle_value(m, n);
  };
  out.assign(twid_count(g), make_float2(0.f, 0.f));
  table(g.nh, out.data());
  table(g.nf, out.data() + g.nh);
  if (g.nfm < 2) return;
  std::vector<std::vector<float2>> mt((size_t)g.nfm);
  for (int d = 0; d < g.nfm; ++d) {
    mt[(size_t)d].resize((size_t)g.fdim[d]);
    table(g.fdim[d], mt[(size_t)d].data());
  }
  float2* fm = out.data() + g.nh + g.nf;
  for (int o = 0; o < g.nf; ++o)
    for (int f = 0; f < g.nf; ++f) {
      double re = 1.0, im = 0.0;
      int ro = o, rf = f;
      for (int d = 0; d < g.nfm; ++d) {
        const int n = g.fdim[d], od = ro % n, fd = rf % n;
        ro /= n;
        rf /= n;
        const float2 w = mt[(size_t)d][(size_t)((od * fd) % n)];
        const double nr = re * w.x - im * w.y, ni = re * w.y + im * w.x;
        re = nr;
        im = ni;
      }
      fm[(size_t)o * g.nf + f] = make_float2((float)re, (float)im);
    }
  int* fp = reinterpret_cast<int*>(fm + (size_t)g.nf * g.nf);
  for (int kf = 0; kf < g.nf; ++kf) fp[kf] = full_partner(g, kf);
}

// Stored slice that holds full-spectrum slice (kf, kfull) itself or its conjugate.
int stored_slice_of(const TubeGeom& g, int kf, int kfull) {
  int f = kf, h = kfull;
  if (h >= g.hh) {  // conjugate partner (-kf, -kh)
    f = full_partner(g, kf);
    h = g.nh - kfull;
  }
  if (!slice_is_distinct(g, f, h)) f = full_partner(g, f);
  return f + g.nf * h;
}

// Number of full-spectrum slices a distinct stored slice stands for (1 or 2).
int slice_weight(const TubeGeom& g, int kf, int kh) {
  const bool selfcol = (kh == 0) || (2 * kh == g.nh);
  const bool selfrow = full_partner(g, kf) == kf;
  return (selfcol && selfrow) ? 1 : 2;
}

int vform_of(const tsvd_ctx* c) { return (c->opts.accumulate_v || c->vform_now) ? 1 : 0; }

std::array<int, 4> plan_key(const Problem& p, int nslices, int vform) {
  return {(int)p.n1, (int)p.n2, nslices, vform};
}
std::array<int, 4> plan_key(tsvd_ctx* c, const Problem& p, int nslices) {
  return plan_key(p, nslices, vform_of(c));
}

// Slice-SVT plans the autotuner compares (or the single plan fixed by the options).
std::vector<SliceKnobs> candidate_knobs(tsvd_ctx* c, const Problem& p, int nslices) {
  const int form = c->opts.slice_form;
  const SliceKnobs base = {c->opts.ctas_per_slice, c->opts.lanes_per_pair, 0, vform_of(c),
                           form == TSVD_SLICE_BLOCK ? 1 : 0};
  std::vector<SliceKnobs> out;
  if (c->opts.autotune) {
    const int ctas[4] = {1, 2, 4, 8};
    const int lanes[4] = {4, 8, 16, 32};
    for (int C : ctas) {
      if (base.ctas && C != base.ctas) continue;
      for (int L : lanes) {
        if (base.lanes && L != base.lanes) continue;
        for (int np = 1; np <= 2 && form != TSVD_SLICE_BLOCK; ++np) {
          const SliceKnobs k = {C, L, np, base.vform, 0};
          if (jacobi_svt_plan_ok((int)p.n1, (int)p.n2, nslices, k)) out.push_back(k);
        }
      }
      // the block form (no lane layout)
      const SliceKnobs kb = {C, 0, 1, base.vform, 1};
      if (form != TSVD_SLICE_PAIRWISE && jacobi_svt_plan_ok((int)p.n1, (int)p.n2, nslices, kb))
        out.push_back(kb);
    }
  }
  if (out.empty()) out.push_back(base);
  return out;
}

// The plan a slice-SVT launch uses: the tuned one when there is one, else the options.
SliceKnobs planned_knobs(tsvd_ctx* c, const Problem& p, int nslices, int vform) {
  auto it = c->tuned.find(plan_key(p, nslices, vform));
  if (it != c->tuned.end()) return it->second;
  return {c->opts.ctas_per_slice, c->opts.lanes_per_pair, 0, vform,
          c->opts.slice_form == TSVD_SLICE_BLOCK ? 1 : 0};
}
SliceKnobs planned_knobs(tsvd_ctx* c, const Problem& p, int nslices) {
  return planned_knobs(c, p, nslices, vform_of(c));
}

std::string device_name(int dev) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string s = prop.name;
  std::replace(s.begin(), s.end(), ' ', '_');
  return s;
}

// Autotune cache file: one line per plan,
// "<gpu> <n1> <n2> <slices> <vform> <ctas> <lanes> <pairs in flight> <block form>".
void load_tune_cache(tsvd_ctx* c) {
  c->cache_loaded = true;
  if (!c->opts.autotune_cache) return;
  FILE* f = std::fopen(c->opts.autotune_cache, "r");
  if (!f) return;
  const std::string me = device_name(c->device);
  char gpu[256];
  int n1, n2, ns, vf, C, L, np, bl;
  while (std::fscanf(f, "%255s %d %d %d %d %d %d %d %d", gpu, &n1, &n2, &ns, &vf, &C, &L, &np,
                     &bl) == 9) {
    const SliceKnobs k = {C, L, np, vf, bl};
    if (me == gpu && jacobi_svt_plan_ok(n1, n2, ns, k)) c->tuned[{n1, n2, ns, vf}] = k;
  }
  std::fclose(f);
}

void store_tune_cache(tsvd_ctx* c, const std::array<int, 4>& key, const SliceKnobs& k) {
  if (!c->opts.autotune_cache) return;
  FILE* f = std::fopen(c->opts.autotune_cache, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %d %d %d %d\n", device_name(c->device).c_str(), key[0],
               key[1], key[2], key[3], k.ctas, k.lanes, k.ppg, k.block);
  std::fclose(f);
}

// Device workspace carved from one allocation.
struct Workspace {
  float2* spec_a = nullptr;
  float2* spec_b = nullptr;
  float* state = nullptr;
  float* yn = nullptr;
  float* stage_in = nullptr;
  uint8_t* stage_om = nullptr;
  float* stage_out0 = nullptr;
  float* stage_out1 = nullptr;
  float2* twid = nullptr;
  int* slices = nullptr;
  SliceStat* stat = nullptr;
  SweepAccum* acc = nullptr;
  int* bad = nullptr;
  void* jscratch = nullptr;     // multi-CTA slice SVT scratch
  size_t jscratch_bytes = 0;
  int ndistinct = 0;
  // mixed form (randomized slice SVT): working matrix Aw = the slice (n1 >= n2) or its
  // transpose, mw x nw with nw <= mw, and its buffers (see RsvtArgs)
  bool rsvt = false;
  int mw = 0, nw = 0, kmax = 0;
  int64_t wr = 0, wc = 0;
  float2 *rP = nullptr, *rY = nullptr, *rQ = nullptr, *rBt = nullptr, *rDt = nullptr,
         *rG = nullptr, *rT = nullptr;
  float* rsig = nullptr;
  unsigned char* risreal = nullptr;
  RsvtStat* rstat = nullptr;     // tsvd_ctx::kRing slots
  void* rjs = nullptr;
  size_t rjs_bytes = 0;
  // plain form, warm start: pre-rotated slices and the accumulated right rotations
  bool warm = false;
  int nv = 0;                    // min(n1, n2)
  float2* abar = nullptr;        // nstore slices like the spectrum
  float2* vwarm = nullptr;       // nstore x nv x nv
};

struct WsRequest {
  bool state = false, yn = false, stage_in = false, stage_om = false, stage_out0 = false,
       stage_out1 = false;
  bool rsvt = false;
  bool warm = false;
};

int rsvt_engine(const tsvd_ctx* c) {
  switch (c->opts.precision) {
    case TSVD_PRECISION_TF32: return RSVT_GEMM_TF32;
    case TSVD_PRECISION_BF16: return RSVT_GEMM_BF16;
    case TSVD_PRECISION_3XTF32: return RSVT_GEMM_3XTF32;
    default: return RSVT_GEMM_FP32;
  }
}

// Noise floor of the slice products relative to sigma_max: singular values below it are
// rounding noise of the products and do not count toward the rank the sketch must cover.
float rsvt_floor(const tsvd_ctx* c) {
  switch (rsvt_engine(c)) {
    case RSVT_GEMM_TF32: return 2e-3f;
    case RSVT_GEMM_BF16: return 1.6e-2f;
    default: return 3e-6f;
  }
}

// Plan of the mixed form's small Jacobi SVTs: the context's fixed choices, else the planner's.
SliceKnobs rsvt_knobs(const tsvd_ctx* c) {
  return {c->opts.ctas_per_slice, c->opts.lanes_per_pair, 0, 0};
}

// A stored slice is real when it is its own conjugate partner.
bool slice_is_real(const TubeGeom& g, int kf, int kh) {
  const bool fh = kh == 0 || 2 * kh == g.nh;
  const bool ff = full_partner(g, kf) == kf;
  return fh && ff;
}

tsvd_status prepare_workspace(tsvd_ctx* c, const Problem& p, const WsRequest& rq, Workspace& w) {
  const TubeGeom& g = p.g;
  const size_t spec = align_up((size_t)g.nstore * g.N12 * sizeof(float2));
  const size_t real = align_up((size_t)p.N * sizeof(float));
  c->slices_host.clear();
  for (int kh = 0; kh < g.hh; ++kh)
    for (int kf = 0; kf < g.nf; ++kf)
      if (slice_is_distinct(g, kf, kh)) c->slices_host.push_back(kf + g.nf * kh);
  w.ndistinct = (int)c->slices_host.size();
  // scratch for every plan the autotuner may try (or for the one fixed plan)
  size_t jbytes = 0;
  if (!rq.rsvt)
    for (const SliceKnobs& k : candidate_knobs(c, p, w.ndistinct))
      jbytes = std::max(jbytes, jacobi_svt_scratch_bytes((int)p.n1, (int)p.n2, w.ndistinct, k));
  // mixed form: orientation and sketch buffers
  w.rsvt = rq.rsvt;
  if (rq.rsvt) {
    const bool tr = p.n1 < p.n2;
    w.mw = (int)(tr ? p.n2 : p.n1);
    w.nw = (int)(tr ? p.n1 : p.n2);
    w.wr = tr ? p.n1 : 1;
    w.wc = tr ? 1 : p.n1;
    w.kmax = std::min(w.nw, rsvt_max_k());
    if (c->opts.rsvt_kmax > 0) w.kmax = std::min(w.kmax, c->opts.rsvt_kmax);
  }
  const size_t ns = (size_t)g.nstore, km = (size_t)w.kmax;
  const size_t rs_nw = rq.rsvt ? ns * w.nw * km * sizeof(float2) : 0;
  const size_t rs_mw = rq.rsvt ? ns * w.mw * km * sizeof(float2) : 0;
  const size_t rs_kk = rq.rsvt ? ns * km * km * sizeof(float2) : 0;
  const size_t rjs = rq.rsvt ? rsvt_jacobi_scratch_bytes(w.nw, w.kmax, w.ndistinct, rsvt_knobs(c)) : 0;
  const size_t warm_v = rq.warm ? ns * (size_t)std::min(p.n1, p.n2) * std::min(p.n1, p.n2) *
                                       sizeof(float2) : 0;
  size_t off[28], total = 0;
  auto take = [&](int i, size_t bytes) { off[i] = total; total += align_up(bytes); };
  take(0, spec);
  take(1, spec);
  take(2, rq.state ? real : 0);
  take(3, rq.yn ? real : 0);
  take(4, rq.stage_in ? real : 0);
  take(5, rq.stage_om ? (size_t)p.N : 0);
  take(6, rq.stage_out0 ? real : 0);
  take(7, rq.stage_out1 ? real : 0);
  take(8, twid_count(g) * sizeof(float2));
  take(9, (size_t)g.nstore * sizeof(int));
  take(10, (size_t)g.nstore * sizeof(SliceStat));
  take(11, sizeof(SweepAccum));
  take(12, sizeof(int));
  take(13, jbytes);
  take(14, rs_nw);   // P
  take(15, rs_mw);   // Y
  take(16, rs_mw);   // Q
  take(17, rs_nw);   // Bt
  take(18, rs_nw);   // Dt
  take(19, rs_kk);   // G
  take(20, rs_kk);   // T
  take(21, rq.rsvt ? ns * km * sizeof(float) : 0);                  // sig
  take(22, rq.rsvt ? ns : 0);                                       // isreal
  take(23, rq.rsvt ? tsvd_ctx::kRing * sizeof(RsvtStat) : 0);       // per-iteration stats
  take(24, rjs);
  take(25, rq.warm ? spec : 0);
  take(26, warm_v);
  if (total > c->ws_cap) {
    if (c->ws) {
      TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
      cudaFree(c->ws);
      c->ws = nullptr;
      c->ws_cap = 0;
      // graphs captured on the old workspace must not replay
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
      c->graphs.clear();
    }
    void* ptr = nullptr;
    cudaError_t e = device_alloc(&ptr, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, TSVD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", total, cudaGetErrorString(e));
    }
    c->ws = static_cast<char*>(ptr);
    c->ws_cap = total;
  }
  char* b = c->ws;
  w.spec_a = reinterpret_cast<float2*>(b + off[0]);
  w.spec_b = reinterpret_cast<float2*>(b + off[1]);
  w.state = rq.state ? reinterpret_cast<float*>(b + off[2]) : nullptr;
  w.yn = rq.yn ? reinterpret_cast<float*>(b + off[3]) : nullptr;
  w.stage_in = rq.stage_in ? reinterpret_cast<float*>(b + off[4]) : nullptr;
  w.stage_om = rq.stage_om ? reinterpret_cast<uint8_t*>(b + off[5]) : nullptr;
  w.stage_out0 = rq.stage_out0 ? reinterpret_cast<float*>(b + off[6]) : nullptr;
  w.stage_out1 = rq.stage_out1 ? reinterpret_cast<float*>(b + off[7]) : nullptr;
  w.twid = reinterpret_cast<float2*>(b + off[8]);
  w.slices = reinterpret_cast<int*>(b + off[9]);
  w.stat = reinterpret_cast<SliceStat*>(b + off[10]);
  w.acc = reinterpret_cast<SweepAccum*>(b + off[11]);
  w.bad = reinterpret_cast<int*>(b + off[12]);
  w.jscratch = jbytes ? b + off[13] : nullptr;
  w.jscratch_bytes = jbytes;
  w.warm = rq.warm;
  w.nv = (int)std::min(p.n1, p.n2);
  w.abar = rq.warm ? reinterpret_cast<float2*>(b + off[25]) : nullptr;
  w.vwarm = rq.warm ? reinterpret_cast<float2*>(b + off[26]) : nullptr;
  if (rq.rsvt) {
    w.rP = reinterpret_cast<float2*>(b + off[14]);
    w.rY = reinterpret_cast<float2*>(b + off[15]);
    w.rQ = reinterpret_cast<float2*>(b + off[16]);
    w.rBt = reinterpret_cast<float2*>(b + off[17]);
    w.rDt = reinterpret_cast<float2*>(b + off[18]);
    w.rG = reinterpret_cast<float2*>(b + off[19]);
    w.rT = reinterpret_cast<float2*>(b + off[20]);
    w.rsig = reinterpret_cast<float*>(b + off[21]);
    w.risreal = reinterpret_cast<unsigned char*>(b + off[22]);
    w.rstat = reinterpret_cast<RsvtStat*>(b + off[23]);
    w.rjs = rjs ? b + off[24] : nullptr;
    w.rjs_bytes = rjs;
    c->isreal_host.assign(ns, 0);
    for (int kh = 0; kh < g.hh; ++kh)
      for (int kf = 0; kf < g.nf; ++kf)
        c->isreal_host[(size_t)(kf + g.nf * kh)] = slice_is_real(g, kf, kh) ? 1 : 0;
    TSVD_CUDA(c, cudaMemcpyAsync(w.risreal, c->isreal_host.data(), ns, cudaMemcpyHostToDevice,
                                 c->stream));
    TSVD_CUDA(c, cudaMemsetAsync(w.rstat, 0, tsvd_ctx::kRing * sizeof(RsvtStat), c->stream));
  }

  fill_twiddles(g, c->twid_host);
  TSVD_CUDA(c, cudaMemcpyAsync(w.twid, c->twid_host.data(), c->twid_host.size() * sizeof(float2),
                               cudaMemcpyHostToDevice, c->stream));
  TSVD_CUDA(c, cudaMemcpyAsync(w.slices, c->slices_host.data(),
                               c->slices_host.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
  TSVD_CUDA(c, cudaMemsetAsync(w.acc, 0, sizeof(SweepAccum), c->stream));
  TSVD_CUDA(c, cudaMemsetAsync(w.stat, 0, (size_t)g.nstore * sizeof(SliceStat), c->stream));
  TSVD_CUDA(c, cudaMemsetAsync(w.bad, 0, sizeof(int), c->stream));
  // The host tables above are pageable; cudaMemcpyAsync from pageable memory returns only
  // after the source has been consumed, so they may change on the next call.
  return TSVD_OK;
}

TubeArgs tube_args(const Problem& p, const Workspace& w, int mode) {
  TubeArgs a{};
  a.g = p.g;
  a.mode = mode;
  a.twid_h = w.twid;
  a.twid_f = w.twid + p.g.nh;
  if (p.g.nfm >= 2) {
    a.fmat = w.twid + p.g.nh + p.g.nf;
    a.fpart = reinterpret_cast<const int*>(w.twid + p.g.nh + p.g.nf + (size_t)p.g.nf * p.g.nf);
  }
  a.ratio = 1.f;
  return a;
}

SliceArgs slice_args(tsvd_ctx* c, const Problem& p, const Workspace& w, float tau) {
  SliceArgs s{};
  s.ahat = w.spec_a;
  s.zhat = w.spec_b;
  s.slices = w.slices;
  s.nslices = w.ndistinct;
  s.n1 = (int)p.n1;
  s.n2 = (int)p.n2;
  s.N12 = p.g.N12;
  s.tau = tau;
  s.tol = c->opts.jacobi_tol;
  s.max_sweeps = c->opts.max_sweeps;
  s.stat = w.stat;
  s.acc = w.acc;
  s.scratch = w.jscratch;
  s.scratch_bytes = w.jscratch_bytes;
  s.knobs = planned_knobs(c, p, w.ndistinct);
  s.abs_stop = c->opts.jacobi_stop == TSVD_STOP_SVT ? 1 : 0;
  return s;
}

// Autotuner: before the first slice-SVT launch of a new (shape, slices, form) in this
// context, time every candidate plan on the current input spectrum (two launches each, the
// second timed, sweeps capped at 4 so that the comparison is per sweep), keep the fastest.
// The candidates write the output spectrum, which the real launch then overwrites.
tsvd_status tune_slices(tsvd_ctx* c, const Problem& p, const Workspace& w, float tau) {
  if (!c->opts.autotune) return TSVD_OK;
  if (!c->cache_loaded) load_tune_cache(c);
  const std::array<int, 4> key = plan_key(c, p, w.ndistinct);
  if (c->tuned.count(key)) return TSVD_OK;
  const std::vector<SliceKnobs> cands = candidate_knobs(c, p, w.ndistinct);
  if (cands.size() == 1) {
    c->tuned[key] = cands[0];
    return TSVD_OK;
  }
  cudaEvent_t e0, e1;
  TSVD_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, TSVD_ECUDA, "cudaEventCreate failed");
  }
  float best = 1e30f;
  SliceKnobs best_k = cands[0];
  for (const SliceKnobs& k : cands) {
    SliceArgs s = slice_args(c, p, w, tau);
    s.knobs = k;
    s.max_sweeps = std::min(4, c->opts.max_sweeps);
    s.stat = nullptr;
    s.acc = nullptr;
    cudaError_t e = launch_jacobi_svt(s, c->stream);
    if (e == cudaSuccess) {
      ++c->launches;
      cudaEventRecord(e0, c->stream);
      e = launch_jacobi_svt(s, c->stream);
      cudaEventRecord(e1, c->stream);
    }
    if (e != cudaSuccess) {   // a plan the device cannot launch (e.g. cluster resources)
      cudaGetLastError();
      continue;
    }
    ++c->launches;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        ms < best) {
      best = ms;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TSVD_CUDA(c, cudaGetLastError());
  c->tuned[key] = best_k;
  store_tune_cache(c, key, best_k);
  return TSVD_OK;
}

double threshold_scale(tsvd_ctx* c, const Problem& p) {
  return c->opts.tnn_scale == TSVD_SCALE_SUM ? (double)p.nslices : 1.0;
}

tsvd_status check_opts(tsvd_ctx* c, const tsvd_opts& o) {
  if (o.precision < TSVD_PRECISION_FP32 || o.precision > TSVD_PRECISION_RAND_FP32)
    return fail(c, TSVD_EINVAL, "bad precision %d", o.precision);
  if (o.rsvt_oversample < 0 || o.rsvt_oversample > 64)
    return fail(c, TSVD_EINVAL, "rsvt_oversample must be in [0, 64]");
  if (o.rsvt_kmax < 0) return fail(c, TSVD_EINVAL, "rsvt_kmax must be >= 0");
  if (o.rsvt_power < 0 || o.rsvt_power > 8) return fail(c, TSVD_EINVAL, "rsvt_power must be in [0, 8]");
  if (o.warm_start != TSVD_WARM_OFF && o.warm_start != TSVD_WARM_ON &&
      o.warm_start != TSVD_WARM_AUTO)
    return fail(c, TSVD_EINVAL, "warm_start must be TSVD_WARM_OFF, _ON or _AUTO");
  if (o.sparse_mode != TSVD_SPARSE_ENTRY && o.sparse_mode != TSVD_SPARSE_TUBE)
    return fail(c, TSVD_EINVAL, "bad sparse_mode %d", o.sparse_mode);
  if (o.tnn_scale != TSVD_SCALE_AVG && o.tnn_scale != TSVD_SCALE_SUM)
    return fail(c, TSVD_EINVAL, "bad tnn_scale %d", o.tnn_scale);
  if (!(o.rho0 > 0) || !std::isfinite(o.rho0) || !(o.mu >= 1) || !std::isfinite(o.mu) ||
      !(o.rho_max >= o.rho0))
    return fail(c, TSVD_EINVAL, "bad penalty schedule (rho0 > 0, mu >= 1, rho_max >= rho0)");
  if (o.max_sweeps < 1) return fail(c, TSVD_EINVAL, "max_sweeps must be >= 1");
  if (!(o.jacobi_tol > 0) || !std::isfinite(o.jacobi_tol))
    return fail(c, TSVD_EINVAL, "jacobi_tol must be positive");
  if (o.ctas_per_slice != 0 && o.ctas_per_slice != 1 && o.ctas_per_slice != 2 &&
      o.ctas_per_slice != 4 && o.ctas_per_slice != 8 && o.ctas_per_slice != TSVD_CTAS_FEWEST)
    return fail(c, TSVD_EINVAL, "ctas_per_slice must be 0, 1, 2, 4, 8 or TSVD_CTAS_FEWEST");
  if (o.accumulate_v != 0 && o.accumulate_v != 1)
    return fail(c, TSVD_EINVAL, "accumulate_v must be 0 or 1");
  if (o.lanes_per_pair != 0 && o.lanes_per_pair != 4 && o.lanes_per_pair != 8 &&
      o.lanes_per_pair != 16 && o.lanes_per_pair != 32)
    return fail(c, TSVD_EINVAL, "lanes_per_pair must be 0, 4, 8, 16 or 32");
  if (o.autotune != 0 && o.autotune != 1) return fail(c, TSVD_EINVAL, "autotune must be 0 or 1");
  if (o.use_graphs != 0 && o.use_graphs != 1)
    return fail(c, TSVD_EINVAL, "use_graphs must be 0 or 1");
  if (o.batch_persistent != 0 && o.batch_persistent != 1)
    return fail(c, TSVD_EINVAL, "batch_persistent must be 0 or 1");
  if (o.rsvt_small_fp64 != 0 && o.rsvt_small_fp64 != 1)
    return fail(c, TSVD_EINVAL, "rsvt_small_fp64 must be 0 or 1");
  if (o.jacobi_stop != TSVD_STOP_SVT && o.jacobi_stop != TSVD_STOP_RELATIVE)
    return fail(c, TSVD_EINVAL, "jacobi_stop must be TSVD_STOP_SVT or TSVD_STOP_RELATIVE");
  if (o.slice_form != TSVD_SLICE_AUTO && o.slice_form != TSVD_SLICE_PAIRWISE &&
      o.slice_form != TSVD_SLICE_BLOCK)
    return fail(c, TSVD_EINVAL, "slice_form must be TSVD_SLICE_AUTO, _PAIRWISE or _BLOCK");
  return TSVD_OK;
}

// Fill host-side result summaries from the per-slice stats of the last t-SVT.
tsvd_status read_slice_stats(tsvd_ctx* c, const Problem& p, const Workspace& w, int32_t* multirank,
                             double* tnn, int* rank_max, bool* all_converged) {
  const TubeGeom& g = p.g;
  c->stat_host.resize((size_t)g.nstore);
  TSVD_CUDA(c, cudaMemcpyAsync(c->stat_host.data(), w.stat, (size_t)g.nstore * sizeof(SliceStat),
                               cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  double t = 0;
  int rmax = 0;
  bool conv = true;
  for (int kh = 0; kh < g.hh; ++kh)
    for (int kf = 0; kf < g.nf; ++kf) {
      if (!slice_is_distinct(g, kf, kh)) continue;
      const SliceStat& st = c->stat_host[(size_t)(kf + g.nf * kh)];
      t += slice_weight(g, kf, kh) * st.nuc;
      if (st.rank > rmax) rmax = st.rank;
      if (!st.converged) conv = false;
    }
  if (multirank) {
    for (int kfull = 0; kfull < g.nh; ++kfull)
      for (int kf = 0; kf < g.nf; ++kf)
        multirank[kf + g.nf * kfull] = c->stat_host[(size_t)stored_slice_of(g, kf, kfull)].rank;
  }
  if (tnn) *tnn = t;
  if (rank_max) *rank_max = rmax;
  if (all_converged) *all_converged = conv;
  return TSVD_OK;
}

tsvd_status launch(tsvd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorInvalidValue)
    return fail(c, TSVD_EUNSUPPORTED, "%s: shape not supported by the kernel", what);
  if (e != cudaSuccess) return fail(c, TSVD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  ++c->launches;
  return TSVD_OK;
}

#define TSVD_TRY(expr)                 \
  do {                                 \
    tsvd_status s_ = (expr);           \
    if (s_ != TSVD_OK) return s_;      \
  } while (0)

void begin_call(tsvd_ctx* c) {
  c->cur = c->stream;
  c->vform_now = false;
  c->err.clear();
  c->launches = 0;
  c->slice_launches = 0;
  c->events_used = 0;
}

// Records one event of a timed pair (opts.timing); kind 0 = slice SVT, 1 = tube pass.
tsvd_status record_event(tsvd_ctx* c, int kind) {
  if (!c->opts.timing) return TSVD_OK;
  if (c->events_used == c->events.size()) {
    cudaEvent_t ev;
    TSVD_CUDA(c, cudaEventCreate(&ev));
    c->events.push_back(ev);
    c->event_kind.push_back(kind);
  }
  c->event_kind[c->events_used] = kind;
  // while capturing, an ordinary record only marks a dependency; an external record becomes
  // an event node of the graph, re-recorded at every replay
  if (c->capturing)
    TSVD_CUDA(c, cudaEventRecordWithFlags(c->events[c->events_used++], c->cur,
                                          cudaEventRecordExternal));
  else
    TSVD_CUDA(c, cudaEventRecord(c->events[c->events_used++], c->cur));
  return TSVD_OK;
}

// Launch helpers: they enqueue on c->cur, which is the context's stream or, while a solver's
// launch sequence is being captured into a graph, the private capture stream.
tsvd_status run_tube(tsvd_ctx* c, const TubeArgs& a, const char* what) {
  NvtxRange nr(what);
  TSVD_TRY(record_event(c, 1));
  TSVD_TRY(launch(c, launch_tube_pass(a, c->cur), what));
  return record_event(c, 1);
}

tsvd_status run_slice(tsvd_ctx* c, const SliceArgs& a) {
  NvtxRange nr("slice SVT (Jacobi)");
  TSVD_TRY(record_event(c, 0));
  TSVD_TRY(launch(c, launch_jacobi_svt(a, c->cur), "slice SVT"));
  ++c->slice_launches;
  return record_event(c, 0);
}

// ---- plain form with warm start
constexpr int kColdEvery = kWarmColdEvery;   // iterations between cold starts of the warm start

// Whether the V form (needed by the warm start) has a plan for this slice shape.
bool warm_plan_exists(tsvd_ctx* c, const Problem& p) {
  const SliceKnobs k = {c->opts.ctas_per_slice, c->opts.lanes_per_pair, 0, 1,
                        c->opts.slice_form == TSVD_SLICE_BLOCK ? 1 : 0};
  return jacobi_svt_plan_ok((int)p.n1, (int)p.n2, p.g.nstore, k);
}

// Plain slice SVT of ADMM iteration `it`.  With the warm start every slice keeps its
// accumulated right rotations V: a warm iteration pre-rotates the slice to B V (vectors as
// columns) or V^T B (vectors as rows) with an FP32 product and starts the Jacobi rotations
// from V; every kColdEvery-th iteration starts from B and V = I (bounding the drift of V).
// The rebuild reads B itself (U form), so neither the FP32 pre-rotation nor a V that is
// unitary only to rounding reaches D_tau(B); they only change how many sweeps converge.
// `kn` (nullable) overrides the context's plan for the shape (a batched tensor's own plan).
tsvd_status plain_slice_step(tsvd_ctx* c, const Problem& p, const Workspace& w, float tau, int it,
                             const SliceKnobs* kn = nullptr) {
  SliceArgs s = slice_args(c, p, w, tau);
  if (kn) s.knobs = *kn;
  if (w.warm) {
    const int nv = w.nv, n1 = (int)p.n1, n2 = (int)p.n2;
    s.vout = w.vwarm;
    s.vstride = (int64_t)nv * nv;
    s.brb = w.spec_a;   // U-form rebuild from B: V only seeds the next iteration
    if (it % kColdEvery != 0) {
      CGemm g{};
      g.batch = w.ndistinct;
      g.M = n1;
      g.N = n2;
      const bool rows = n1 < n2;   // the Jacobi vectors are the rows of the slice
      g.K = rows ? n1 : n2;
      // A(i, l): the slice (columns) or V^T (rows); B(l, j): V (columns) or the slice (rows)
      const CMat slice_m = {w.spec_a, w.slices, p.g.N12, 1, (int64_t)n1, 0};
      const CMat v_m = {w.vwarm, w.slices, (int64_t)nv * nv, 1, (int64_t)nv, 0};
      const CMat vt_m = {w.vwarm, w.slices, (int64_t)nv * nv, (int64_t)nv, 1, 0};
      g.a = rows ? vt_m : slice_m;
      g.b = rows ? slice_m : v_m;
      g.c = {w.abar, w.slices, p.g.N12, 1, (int64_t)n1, 0};
      TSVD_TRY(launch(c, launch_cgemm(g, RSVT_GEMM_FP32, c->cur), "warm-start rotation"));
      s.ahat = w.abar;
      s.vin = w.vwarm;
    }
  }
  return run_slice(c, s);
}

// ---- mixed form: randomized slice SVT
RsvtArgs rsvt_args(tsvd_ctx* c, const Problem& p, const Workspace& w, float tau, int k,
                   int iter) {
  RsvtArgs a{};
  a.ahat = w.spec_a;
  a.zhat = w.spec_b;
  a.slices = w.slices;
  a.nslices = w.ndistinct;
  a.mw = w.mw;
  a.nw = w.nw;
  a.wr = w.wr;
  a.wc = w.wc;
  a.N12 = p.g.N12;
  a.k = k;
  a.kmax = w.kmax;
  a.kfill = w.kmax;
  a.power = 0;
  a.tau = tau;
  a.floor_rel = rsvt_floor(c);
  a.chol_tol = 1e-5f;
  a.tol = c->opts.jacobi_tol;
  a.max_sweeps = c->opts.max_sweeps;
  a.seed = 0x7473766473656564ull;
  a.iter = iter;
  a.engine = rsvt_engine(c);
  a.stat = w.stat;
  a.acc = w.acc;
  a.rstat = w.rstat + (iter % tsvd_ctx::kRing);
  a.P = w.rP;
  a.Y = w.rY;
  a.Q = w.rQ;
  a.Bt = w.rBt;
  a.Dt = w.rDt;
  a.G = w.rG;
  a.T = w.rT;
  a.sig = w.rsig;
  a.isreal = w.risreal;
  a.jscratch = w.rjs;
  a.jscratch_bytes = w.rjs_bytes;
  a.jknobs = rsvt_knobs(c);
  a.small_fp64 = c->opts.rsvt_small_fp64;
  a.abs_stop = c->opts.jacobi_stop == TSVD_STOP_SVT ? 1 : 0;
  return a;
}

// Kernels one launch_rsvt call enqueues.
int rsvt_kernels(const RsvtArgs& a) {
  return 8 * (a.power + 1) + 3 + (a.k <= rsvt_eig_max_k() ? 3 : 0);
}

// Smallest sketch width: the oversampling margin over rank 8, rounded up to 8.
int rsvt_k0(const tsvd_ctx* c, const Workspace& w) {
  const int k = (8 + c->opts.rsvt_oversample + 7) / 8 * 8;
  return std::max(1, std::min(k, w.kmax));
}

int rsvt_k_for(const tsvd_ctx* c, const Workspace& w, int rank) {
  const int k = (rank + c->opts.rsvt_oversample + 7) / 8 * 8;
  return std::max(1, std::min(k, w.kmax));
}

tsvd_status rsvt_host_ring(tsvd_ctx* c) {
  if (c->rs_host) return TSVD_OK;
  void* h = nullptr;
  TSVD_CUDA(c, cudaMallocHost(&h, tsvd_ctx::kRing * sizeof(RsvtStat)));
  c->rs_host = static_cast<RsvtStat*>(h);
  std::memset(c->rs_host, 0, tsvd_ctx::kRing * sizeof(RsvtStat));
  for (int i = 0; i < tsvd_ctx::kRing; ++i)
    TSVD_CUDA(c, cudaEventCreateWithFlags(&c->rs_ev[i], cudaEventDisableTiming));
  return TSVD_OK;
}

// Starts a randomized-SVT sequence: random P (all columns), counters reset.
tsvd_status rsvt_begin(tsvd_ctx* c, const Problem& p, const Workspace& w) {
  TSVD_TRY(rsvt_host_ring(c));
  c->rs_k_last = 0;
  c->rs_saturated = c->rs_drops = 0;
  c->rs_gemm_gflop = c->rs_svd_gflop = 0;
  c->rs_stage_used = 0;
  RsvtArgs a = rsvt_args(c, p, w, 0.f, 0, 0);
  a.rstat = nullptr;
  TSVD_TRY(launch(c, launch_rsvt_refill(a, 0, w.kmax, c->cur), "sketch initialisation"));
  return TSVD_OK;
}

// One randomized slice SVT (iteration `iter` of a sequence) with sketch width k; its
// statistics land in ring slot iter % kRing of the host copy, signalled by rs_ev.
tsvd_status rsvt_step(tsvd_ctx* c, const Problem& p, const Workspace& w, float tau, int k,
                      int iter, int power) {
  RsvtArgs a = rsvt_args(c, p, w, tau, k, iter);
  a.power = power;
  const int slot = iter % tsvd_ctx::kRing;
  if (c->opts.timing && power == 0) {
    if (c->rs_stage_used == c->rs_stage.size()) {
      std::array<cudaEvent_t, 7> evs{};
      for (cudaEvent_t& ev : evs) TSVD_CUDA(c, cudaEventCreate(&ev));
      c->rs_stage.push_back(evs);
    }
    a.stage_ev = c->rs_stage[c->rs_stage_used++].data();
  }
  // algorithmic work: three complex products and the GvL count of the small SVDs
  const double mw = w.mw, nw = w.nw, kk = k, ns = w.ndistinct;
  c->rs_gemm_gflop += (power + 1) * ns * 3.0 * 8.0 * mw * nw * kk * 1e-9;
  c->rs_svd_gflop += ns * 4.0 * (4.0 * nw * kk * kk + 8.0 * kk * kk * kk) * 1e-9;
  NvtxRange nr("slice SVT (randomized)");
  TSVD_CUDA(c, cudaMemsetAsync(a.rstat, 0, sizeof(RsvtStat), c->cur));
  TSVD_TRY(record_event(c, 0));
  TSVD_TRY(launch(c, launch_rsvt(a, c->cur), "randomized slice SVT"));
  c->launches += rsvt_kernels(a) - 1;
  ++c->slice_launches;
  TSVD_TRY(record_event(c, 0));
  TSVD_CUDA(c, cudaMemcpyAsync(c->rs_host + slot, a.rstat, sizeof(RsvtStat),
                               cudaMemcpyDeviceToHost, c->cur));
  TSVD_CUDA(c, cudaEventRecord(c->rs_ev[slot], c->cur));
  c->rs_k_last = k;
  return TSVD_OK;
}

// Tensor-core products whose bounded waits expired make the call fail with ETIMEOUT.
tsvd_status rsvt_check_timeouts(tsvd_ctx* c) {
  if (rsvt_engine(c) == RSVT_GEMM_FP32) return TSVD_OK;
  int n = 0;
  TSVD_CUDA(c, tc_gemm_take_timeouts(&n, c->stream));
  if (n) return fail(c, TSVD_ETIMEOUT, "%d tensor-core product launches timed out", n);
  return TSVD_OK;
}

// Waits for the statistics of iteration `iter` and folds them into the call's counters.
tsvd_status rsvt_collect(tsvd_ctx* c, int iter, RsvtStat* out) {
  const int slot = iter % tsvd_ctx::kRing;
  TSVD_CUDA(c, cudaEventSynchronize(c->rs_ev[slot]));
  const RsvtStat s = c->rs_host[slot];
  c->rs_saturated += s.saturated;
  c->rs_drops += s.drops;
  if (out) *out = s;
  return TSVD_OK;
}

// The sketch widths of an ADMM loop: iteration t uses the width chosen from the ranks seen in
// iteration t - 2 (never smaller than the previous width).
struct RsvtLoop {
  tsvd_ctx* c;
  const Problem& p;
  const Workspace& w;
  int k = 0;
  int done = 0;   // iterations whose statistics were collected
  int issued = 0;
  RsvtLoop(tsvd_ctx* c_, const Problem& p_, const Workspace& w_) : c(c_), p(p_), w(w_) {}
  tsvd_status begin() {
    k = rsvt_k0(c, w);
    return rsvt_begin(c, p, w);
  }
  tsvd_status step(float tau) {
    while (done + 2 <= issued) {
      RsvtStat s;
      TSVD_TRY(rsvt_collect(c, done, &s));
      k = std::max(k, rsvt_k_for(c, w, s.rank_max));
      ++done;
    }
    TSVD_TRY(rsvt_step(c, p, w, tau, k, issued, 0));
    ++issued;
    return TSVD_OK;
  }
  tsvd_status finish() {
    while (done < issued) TSVD_TRY(rsvt_collect(c, done++, nullptr));
    return rsvt_check_timeouts(c);
  }
};

// Runs `body` (which only enqueues kernels through the helpers above) directly, or -- when
// graphs are enabled and the launch sequence cannot change (`capturable`: no autotuning or
// host synchronisation left in it) -- replays the CUDA graph cached under `key`, capturing
// it on first use.  Key = everything the launches depend on (buffers, shape, iteration
// count, options, workspace, plan).
template <class F>
tsvd_status run_maybe_graph(tsvd_ctx* c, const std::vector<int64_t>& key, bool capturable,
                            F&& body) {
  c->cur = c->stream;
  if (!c->opts.use_graphs || !capturable) return body();
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (!c->cap_stream)
      TSVD_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (c->graphs.size() >= 8) {   // keep a few recent graphs only
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
      c->graphs.clear();
    }
    const int64_t l0 = c->launches, s0 = c->slice_launches;
    const size_t e0 = c->events_used;
    TSVD_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->cur = c->cap_stream;
    c->capturing = true;
    const tsvd_status st = body();
    c->capturing = false;
    c->cur = c->stream;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
    if (ec != cudaSuccess) cudaGetLastError();   // not left behind for a later launch check
    if (st != TSVD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ec != cudaSuccess) return fail(c, TSVD_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
    tsvd_ctx::Graph g;
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(c, TSVD_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    g.launches = c->launches - l0;
    g.slice_launches = c->slice_launches - s0;
    g.events_used = c->events_used - e0;
    it = c->graphs.emplace(key, g).first;
    c->launches = l0;
    c->slice_launches = s0;
    c->events_used = e0;
  }
  TSVD_CUDA(c, cudaGraphLaunch(it->second.exec, c->stream));
  c->launches += it->second.launches;
  c->slice_launches += it->second.slice_launches;
  c->events_used += it->second.events_used;
  return TSVD_OK;
}

std::vector<int64_t> solver_key(tsvd_ctx* c, int kind, const Problem& p, int iters,
                                std::initializer_list<const void*> ptrs, const SliceKnobs& k) {
  std::vector<int64_t> key = {kind, p.order, p.n1, p.n2, p.n3, p.n4, iters,
                              (int64_t)(intptr_t)c->ws, (int64_t)c->ws_cap, k.ctas, k.lanes,
                              k.ppg, k.vform, c->opts.tnn_scale, c->opts.sparse_mode,
                              c->opts.max_sweeps, c->opts.timing, c->vform_now ? 1 : 0};
  for (const void* q : ptrs) key.push_back((int64_t)(intptr_t)q);
  double d[4] = {c->opts.rho0, c->opts.mu, c->opts.rho_max, (double)c->opts.jacobi_tol};
  for (double v : d) {
    int64_t bits;
    std::memcpy(&bits, &v, sizeof bits);
    key.push_back(bits);
  }
  return key;
}

// Sum of the timed pairs per kind (waits for the stream).
tsvd_status timed_totals(tsvd_ctx* c, double* slice_ms, double* tube_ms) {
  *slice_ms = *tube_ms = 0.0;
  if (!c->opts.timing || c->events_used == 0) return TSVD_OK;
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i + 1 < c->events_used; i += 2) {
    float ms = 0.f;
    TSVD_CUDA(c, cudaEventElapsedTime(&ms, c->events[i], c->events[i + 1]));
    if (c->event_kind[i] == 0) *slice_ms += ms;
    else *tube_ms += ms;
  }
  return TSVD_OK;
}

tsvd_status fill_stats(tsvd_ctx* c, const Problem& p, const Workspace& w, int iters, double rho,
                       tsvd_stats* stats) {
  if (!stats) return TSVD_OK;
  std::memset(stats, 0, sizeof *stats);
  stats->iters = iters;
  stats->rho_final = rho;
  stats->launches = c->launches;
  stats->slice_launches = c->slice_launches;
  if (w.rsvt) {
    stats->slice_ctas =
        c->rs_k_last == 0 ? 0
        : c->rs_k_last <= rsvt_eig_max_k()
            ? 1
            : jacobi_svt_ctas_per_slice(w.nw, c->rs_k_last, w.ndistinct, rsvt_knobs(c));
    stats->rsvt_k_last = c->rs_k_last;
    stats->rsvt_saturated = c->rs_saturated;
    stats->rsvt_drops = c->rs_drops;
    stats->rsvt_gemm_gflop = c->rs_gemm_gflop;
    stats->rsvt_svd_gflop = c->rs_svd_gflop;
    if (c->opts.timing && c->rs_stage_used) {
      TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
      for (size_t i = 0; i < c->rs_stage_used; ++i) {
        const auto& ev = c->rs_stage[i];
        float t[6];
        for (int j = 0; j < 6; ++j) TSVD_CUDA(c, cudaEventElapsedTime(&t[j], ev[j], ev[j + 1]));
        stats->rsvt_gemm_ms += t[0] + t[2] + t[4];
        stats->rsvt_orth_ms += t[1];
        stats->rsvt_svd_ms += t[3];
      }
    }
  } else {
    const SliceKnobs k = planned_knobs(c, p, w.ndistinct);
    stats->slice_ctas = jacobi_svt_ctas_per_slice((int)p.n1, (int)p.n2, w.ndistinct, k);
    stats->slice_lanes = k.lanes;
    stats->slice_pairs_in_flight = k.ppg;
  }
  TSVD_TRY(timed_totals(c, &stats->slice_ms, &stats->tube_ms));
  if (iters <= 0) return TSVD_OK;
  SweepAccum acc;
  TSVD_CUDA(c, cudaMemcpyAsync(&acc, w.acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  int rmax = 0;
  double tnn = 0;
  TSVD_TRY(read_slice_stats(c, p, w, nullptr, &tnn, &rmax, nullptr));
  stats->max_sweeps_used = acc.max_sweeps;
  stats->total_sweeps = (int64_t)acc.total_sweeps;
  stats->nonconverged = (int64_t)acc.nonconverged;
  stats->slice_svds = (int64_t)iters * w.ndistinct;
  stats->tnn_last = tnn;
  stats->rank_last_max = rmax;
  return TSVD_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched solves: one workspace region per tensor, one kernel chain per tensor.
// ---------------------------------------------------------------------------------------------
struct BatchItem {
  const tsvd_problem* src = nullptr;
  Problem p;
  Workspace w;
  SliceKnobs kn{};
  std::vector<float2> twid;
  std::vector<int> slices;
  std::vector<unsigned char> isreal;   // mixed form
  bool warm = false;                   // plain form with the warm-started Jacobi
};

// Carves the regions of one tensor from `base` (nullptr: only measure); returns its bytes.
size_t carve_item(tsvd_ctx* c, BatchItem& it, char* base, int iters, bool persistent = false) {
  const TubeGeom& g = it.p.g;
  it.slices.clear();
  for (int kh = 0; kh < g.hh; ++kh)
    for (int kf = 0; kf < g.nf; ++kf)
      if (slice_is_distinct(g, kf, kh)) it.slices.push_back(kf + g.nf * kh);
  it.w.ndistinct = (int)it.slices.size();
  const size_t spec = (size_t)g.nstore * g.N12 * sizeof(float2);
  const size_t real = (size_t)it.p.N * sizeof(float);
  const bool complete = it.src->kind == TSVD_PROBLEM_COMPLETE;
  const bool mixed = mixed_precision(c);
  // the warm start as in the single-tensor solves
  const int ws = c->opts.warm_start;
  it.warm = !mixed && iters >= 2 && ws != TSVD_WARM_OFF && warm_plan_exists(c, it.p);
  it.kn = planned_knobs(c, it.p, it.w.ndistinct, it.warm ? 1 : vform_of(c));
  // (the persistent batched kernel keeps one exchange buffer per cluster instead)
  const size_t jbytes = mixed || persistent ? 0
                        : jacobi_svt_scratch_bytes((int)it.p.n1, (int)it.p.n2, it.w.ndistinct, it.kn);
  size_t total = 0;
  auto take = [&](size_t bytes) {
    char* ptr = base ? base + total : nullptr;
    total += align_up(bytes);
    return ptr;
  };
  it.w.spec_a = reinterpret_cast<float2*>(take(spec));
  it.w.spec_b = reinterpret_cast<float2*>(take(spec));
  it.w.state = reinterpret_cast<float*>(take(real));
  it.w.yn = complete ? reinterpret_cast<float*>(take(real)) : nullptr;
  it.w.twid = reinterpret_cast<float2*>(take(twid_count(g) * sizeof(float2)));
  it.w.slices = reinterpret_cast<int*>(take((size_t)g.nstore * sizeof(int)));
  it.w.stat = reinterpret_cast<SliceStat*>(take((size_t)g.nstore * sizeof(SliceStat)));
  it.w.acc = reinterpret_cast<SweepAccum*>(take(sizeof(SweepAccum)));
  it.w.jscratch = jbytes ? take(jbytes) : nullptr;
  it.w.jscratch_bytes = jbytes;
  it.w.warm = it.warm;
  it.w.nv = (int)std::min(it.p.n1, it.p.n2);
  if (it.warm) {
    // the persistent kernel forms the pre-rotated slices while loading them
    it.w.abar = persistent ? nullptr : reinterpret_cast<float2*>(take(spec));
    it.w.vwarm = reinterpret_cast<float2*>(
        take((size_t)g.nstore * it.w.nv * it.w.nv * sizeof(float2)));
  }
  it.w.rsvt = mixed;
  if (mixed) {
    // mixed form with the device-chosen width (graph-capturable): widths up to the Gram path's
    const bool tr = it.p.n1 < it.p.n2;
    it.w.mw = (int)(tr ? it.p.n2 : it.p.n1);
    it.w.nw = (int)(tr ? it.p.n1 : it.p.n2);
    it.w.wr = tr ? it.p.n1 : 1;
    it.w.wc = tr ? 1 : it.p.n1;
    it.w.kmax = std::min(it.w.nw, rsvt_eig_max_k());
    if (c->opts.rsvt_kmax > 0) it.w.kmax = std::min(it.w.kmax, c->opts.rsvt_kmax);
    const size_t ns = (size_t)g.nstore, km = (size_t)it.w.kmax;
    it.w.rP = reinterpret_cast<float2*>(take(ns * it.w.nw * km * sizeof(float2)));
    it.w.rY = reinterpret_cast<float2*>(take(ns * it.w.mw * km * sizeof(float2)));
    it.w.rQ = reinterpret_cast<float2*>(take(ns * it.w.mw * km * sizeof(float2)));
    it.w.rBt = reinterpret_cast<float2*>(take(ns * it.w.nw * km * sizeof(float2)));
    it.w.rDt = reinterpret_cast<float2*>(take(ns * it.w.nw * km * sizeof(float2)));
    it.w.rG = reinterpret_cast<float2*>(take(ns * km * km * sizeof(float2)));
    it.w.rT = reinterpret_cast<float2*>(take(ns * km * km * sizeof(float2)));
    it.w.rsig = reinterpret_cast<float*>(take(ns * km * sizeof(float)));
    it.w.risreal = reinterpret_cast<unsigned char*>(take(ns));
    it.w.rstat = reinterpret_cast<RsvtStat*>(take(sizeof(RsvtStat)));
    it.w.rjs = nullptr;
    it.w.rjs_bytes = 0;
    it.isreal.assign(ns, 0);
    for (int kh = 0; kh < g.hh; ++kh)
      for (int kf = 0; kf < g.nf; ++kf)
        it.isreal[(size_t)(kf + g.nf * kh)] = slice_is_real(g, kf, kh) ? 1 : 0;
  }
  return total;
}

// The whole launch chain of one tensor (all iterations) on c->cur.
tsvd_status enqueue_item(tsvd_ctx* c, const BatchItem& it, int iters) {
  const Problem& p = it.p;
  const Workspace& w = it.w;
  const tsvd_problem& q = *it.src;
  const double scale = threshold_scale(c, p);
  double r = c->opts.rho0;
  if (q.kind == TSVD_PROBLEM_COMPLETE) {
    TubeArgs t0 = tube_args(p, w, TUBE_COMPLETE);
    t0.in = w.yn;
    t0.state = w.state;
    t0.spec_out = w.spec_a;
    t0.first = 1;
    t0.write_out = iters == 1;
    t0.out0 = q.out0;
    TSVD_TRY(run_tube(c, t0, "completion pass"));
  } else {
    TubeArgs t0 = tube_args(p, w, TUBE_FWD);
    t0.in = q.M;
    t0.spec_out = w.spec_a;
    TSVD_TRY(run_tube(c, t0, "tube pass (forward)"));
  }
  if (w.rsvt) {
    // device-chosen sketch width: counters and width reset, random start basis
    TSVD_TRY(launch(c, launch_rsvt_state_init(w.rstat, rsvt_k0(c, w), c->cur), "sketch state"));
    RsvtArgs a0 = rsvt_args(c, p, w, 0.f, 0, 0);
    a0.rstat = nullptr;
    TSVD_TRY(launch(c, launch_rsvt_refill(a0, 0, w.kmax, c->cur), "sketch initialisation"));
  }
  for (int k = 0; k < iters; ++k) {
    const float tau = (float)(scale / r);
    if (w.rsvt) {
      RsvtArgs a = rsvt_args(c, p, w, tau, w.kmax, k);
      a.rstat = w.rstat;
      a.kdev = &w.rstat->k;
      a.oversample = c->opts.rsvt_oversample;
      TSVD_TRY(record_event(c, 0));
      TSVD_TRY(launch(c, launch_rsvt(a, c->cur), "randomized slice SVT"));
      c->launches += rsvt_kernels(a);   // + the width update
      ++c->slice_launches;
      TSVD_TRY(record_event(c, 0));
    } else {
      TSVD_TRY(plain_slice_step(c, p, w, tau, k, &it.kn));
    }
    const double r_next = std::fmin(c->opts.mu * r, c->opts.rho_max);
    if (q.kind == TSVD_PROBLEM_COMPLETE) {
      if (k + 1 < iters) {
        TubeArgs t = tube_args(p, w, TUBE_COMPLETE);
        t.in = w.yn;
        t.state = w.state;
        t.spec_in = w.spec_b;
        t.spec_out = w.spec_a;
        t.ratio = (float)(r / r_next);
        t.write_out = (k + 2 == iters);
        t.out0 = q.out0;
        TSVD_TRY(run_tube(c, t, "completion pass"));
      }
    } else {
      TubeArgs t = tube_args(p, w, TUBE_RPCA);
      t.in = q.M;
      t.state = w.state;
      t.spec_in = w.spec_b;
      t.spec_out = w.spec_a;
      t.ratio = (float)(r / r_next);
      t.kappa = (float)((double)q.lambda / r);
      t.first = k == 0;
      t.last = k + 1 == iters;
      t.out0 = q.out0;
      t.out1 = q.out1;
      t.tube_sparse = c->opts.sparse_mode == TSVD_SPARSE_TUBE;
      TSVD_TRY(run_tube(c, t, "RPCA pass"));
    }
    r = r_next;
  }
  if (q.kind == TSVD_PROBLEM_COMPLETE && q.out1) {
    TubeArgs inv = tube_args(p, w, TUBE_INV);
    inv.spec_in = w.spec_b;
    inv.out0 = q.out1;
    TSVD_TRY(run_tube(c, inv, "tube pass (inverse)"));
  }
  return TSVD_OK;
}

}  // namespace

extern "C" {

void tsvd_default_opts(tsvd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = TSVD_PRECISION_FP32;
  o->sparse_mode = TSVD_SPARSE_ENTRY;
  o->tnn_scale = TSVD_SCALE_AVG;
  o->rho0 = 1e-2;
  o->mu = 1.1;
  o->rho_max = 1e10;
  o->max_sweeps = 40;
  o->jacobi_tol = 1e-6f;
  o->autotune = 1;
  o->use_graphs = 1;
  o->rsvt_oversample = 10;
  o->rsvt_kmax = 0;
  o->rsvt_power = 2;
  o->warm_start = TSVD_WARM_AUTO;
  o->batch_persistent = 0;
  o->jacobi_stop = TSVD_STOP_SVT;
}

tsvd_status tsvd_create(tsvd_ctx** out, int device, void* cuda_stream, const tsvd_opts* opts) {
  if (!out) return TSVD_EINVAL;
  *out = nullptr;
  tsvd_ctx* c = new (std::nothrow) tsvd_ctx();
  if (!c) return TSVD_ENOMEM;
  if (opts) c->opts = *opts;
  else tsvd_default_opts(&c->opts);
  tsvd_status st = check_opts(c, c->opts);
  if (st != TSVD_OK) {
    delete c;
    return st;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete c;
    return TSVD_ECUDA;
  }
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = c;
  return TSVD_OK;
}

tsvd_status tsvd_destroy(tsvd_ctx* c) {
  if (!c) return TSVD_OK;
  DeviceGuard dg(c->device);
  tsvd_status st = TSVD_OK;
  if (c->ws) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = TSVD_ECUDA;
    cudaFree(c->ws);
  }
  for (cudaEvent_t ev : c->events) cudaEventDestroy(ev);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaStream_t s : c->branches) cudaStreamDestroy(s);
  for (cudaEvent_t e : c->joins) cudaEventDestroy(e);
  if (c->fork) cudaEventDestroy(c->fork);
  for (cudaEvent_t e : c->rs_ev)
    if (e) cudaEventDestroy(e);
  for (auto& evs : c->rs_stage)
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
  if (c->rs_host) cudaFreeHost(c->rs_host);
  if (c->fbuf) cudaFree(c->fbuf);
  delete c;
  return st;
}

const char* tsvd_last_error(const tsvd_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

tsvd_status tsvt(tsvd_ctx* c, const float* Y, float* Z, int order, const int64_t* dims,
                 float tau, int32_t* multirank, double* tnn) {
  if (!c) return TSVD_EINVAL;
  NvtxRange nr("tsvt");
  begin_call(c);
  if (!Y || !Z) return fail(c, TSVD_EINVAL, "Y and Z must not be NULL");
  if (!(tau >= 0.f) || !std::isfinite(tau)) return fail(c, TSVD_EINVAL, "tau must be finite and >= 0");
  Problem p;
  TSVD_TRY(make_problem(c, order, dims, p));
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int ky = pointer_kind(Y, c->device), kz = pointer_kind(Z, c->device);
  if (ky < 0 || kz < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  WsRequest rq;
  rq.stage_in = ky == 1;
  rq.stage_out0 = kz == 1;
  rq.rsvt = mixed_precision(c);
  Workspace w;
  TSVD_TRY(prepare_workspace(c, p, rq, w));
  const size_t bytes = (size_t)p.N * sizeof(float);
  const float* y = Y;
  float* z = Z;
  if (ky == 1) {
    TSVD_CUDA(c, cudaMemcpyAsync(w.stage_in, Y, bytes, cudaMemcpyHostToDevice, c->stream));
    y = w.stage_in;
  }
  if (kz == 1) z = w.stage_out0;

  TubeArgs f = tube_args(p, w, TUBE_FWD);
  f.in = y;
  f.spec_out = w.spec_a;
  TSVD_TRY(run_tube(c, f, "tube pass (forward)"));
  if (w.rsvt) {
    // random start with power steps; the sketch doubles while the ranks fill it
    TSVD_TRY(rsvt_begin(c, p, w));
    int k = rsvt_k0(c, w);
    for (int attempt = 0;; ++attempt) {
      TSVD_TRY(rsvt_step(c, p, w, tau, k, attempt, c->opts.rsvt_power));
      RsvtStat st;
      TSVD_TRY(rsvt_collect(c, attempt, &st));
      const int need = rsvt_k_for(c, w, st.rank_max);
      if (need <= k || k >= w.kmax) break;
      k = std::min(w.kmax, std::max(need, 2 * k));
    }
    TSVD_TRY(rsvt_check_timeouts(c));
  } else {
    TSVD_TRY(tune_slices(c, p, w, tau));
    SliceArgs s = slice_args(c, p, w, tau);
    TSVD_TRY(run_slice(c, s));
  }
  TubeArgs inv = tube_args(p, w, TUBE_INV);
  inv.spec_in = w.spec_b;
  inv.out0 = z;
  TSVD_TRY(run_tube(c, inv, "tube pass (inverse)"));
  if (kz == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(Z, w.stage_out0, bytes, cudaMemcpyDeviceToHost, c->stream));
  bool conv = true;
  TSVD_TRY(read_slice_stats(c, p, w, multirank, tnn, nullptr, &conv));
  if (!conv) return fail(c, TSVD_ENOTCONV, "a slice SVD reached max_sweeps = %d", c->opts.max_sweeps);
  return TSVD_OK;
}

// The slice SVDs behind tsvd_factor and tsvd_compress: forward tube pass, then the one-sided
// Jacobi of every distinct Fourier slice in the V form (V = I at the start) with a threshold
// above every singular value (its own rebuild keeps nothing), writing the converged vectors W,
// their norms sigma and the rotations J into the context's factor buffer, followed by
// `extra` further bytes for the caller (fw.extra).
struct FactorWork {
  Problem p;
  Workspace w;
  int n1 = 0, n2 = 0, nv = 0, len = 0;
  float2* W = nullptr;
  float2* J = nullptr;
  float* sig = nullptr;
  char* extra = nullptr;
};

// The context's buffer for the factor, compression and t-product calls, grown to `need` bytes
// (the old one is freed after the stream drains).
tsvd_status grow_fbuf(tsvd_ctx* c, size_t need) {
  if (need <= c->fbuf_cap) return TSVD_OK;
  if (c->fbuf) {
    TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->fbuf);
    c->fbuf = nullptr;
    c->fbuf_cap = 0;
  }
  void* ptr = nullptr;
  const cudaError_t e = device_alloc(&ptr, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, TSVD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", need, cudaGetErrorString(e));
  }
  c->fbuf = static_cast<char*>(ptr);
  c->fbuf_cap = need;
  return TSVD_OK;
}

tsvd_status factor_slices(tsvd_ctx* c, const float* Y, int order, const int64_t* dims,
                          size_t extra, FactorWork& fw) {
  Problem& p = fw.p;
  TSVD_TRY(make_problem(c, order, dims, p));
  if (!jacobi_svt_supported((int)p.n1, (int)p.n2))
    return fail(c, TSVD_EUNSUPPORTED, "a %lld x %lld complex slice does not fit one SM's shared memory",
                (long long)p.n1, (long long)p.n2);
  fw.n1 = (int)p.n1;
  fw.n2 = (int)p.n2;
  fw.nv = std::min(fw.n1, fw.n2);
  fw.len = std::max(fw.n1, fw.n2);
  if (!warm_plan_exists(c, p))
    return fail(c, TSVD_EUNSUPPORTED, "no slice plan keeps the rotations of a %d x %d slice",
                fw.n1, fw.n2);
  const int ky = pointer_kind(Y, c->device);
  if (ky < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  // the plans (and the scratch sized for them) are those of the V form
  c->vform_now = true;
  WsRequest rq;
  rq.stage_in = ky == 1;
  TSVD_TRY(prepare_workspace(c, p, rq, fw.w));
  const size_t ns = (size_t)p.g.nstore;
  const size_t b_w = align_up(ns * fw.len * fw.nv * sizeof(float2));
  const size_t b_j = align_up(ns * fw.nv * fw.nv * sizeof(float2));
  const size_t b_s = align_up(ns * fw.nv * sizeof(float));
  TSVD_TRY(grow_fbuf(c, b_w + b_j + b_s + align_up(extra)));
  fw.W = reinterpret_cast<float2*>(c->fbuf);
  fw.J = reinterpret_cast<float2*>(c->fbuf + b_w);
  fw.sig = reinterpret_cast<float*>(c->fbuf + b_w + b_j);
  fw.extra = c->fbuf + b_w + b_j + b_s;
  const float* y = Y;
  if (ky == 1) {
    TSVD_CUDA(c, cudaMemcpyAsync(fw.w.stage_in, Y, (size_t)p.N * sizeof(float),
                                 cudaMemcpyHostToDevice, c->stream));
    y = fw.w.stage_in;
  }
  TubeArgs f = tube_args(p, fw.w, TUBE_FWD);
  f.in = y;
  f.spec_out = fw.w.spec_a;
  TSVD_TRY(run_tube(c, f, "tube pass (forward)"));
  const float tau_none = 3.0e38f;   // keeps no singular value: the slice pass only factors
  TSVD_TRY(tune_slices(c, p, fw.w, tau_none));
  SliceArgs sa = slice_args(c, p, fw.w, tau_none);
  sa.wout = fw.W;
  sa.wout_stride = (int64_t)fw.len * fw.nv;
  sa.sigout = fw.sig;
  sa.sig_stride = fw.nv;
  sa.vout = fw.J;
  sa.vstride = (int64_t)fw.nv * fw.nv;
  sa.abs_stop = 0;   // a factorisation keeps every direction: the relative test alone
  return run_slice(c, sa);
}

FactorArgs factor_args(const FactorWork& fw, int k) {
  FactorArgs fa{};
  fa.W = fw.W;
  fa.sig = fw.sig;
  fa.J = fw.J;
  fa.slices = fw.w.slices;
  fa.nslices = fw.w.ndistinct;
  fa.n1 = fw.n1;
  fa.n2 = fw.n2;
  fa.k = k;
  return fa;
}

// Truncated t-SVD (Algorithm 1, Theorem 2.3.1): the slice SVDs, the Fourier-domain factors
// ordered by decreasing singular value (factor.cu), one inverse tube pass per factor.
tsvd_status tsvd_factor(tsvd_ctx* c, const float* Y, int order, const int64_t* dims, int k,
                        float* U, float* S, float* V) {
  if (!c) return TSVD_EINVAL;
  begin_call(c);
  if (!Y || !U || !S || !V) return fail(c, TSVD_EINVAL, "Y, U, S and V must not be NULL");
  if ((const void*)U == Y || (const void*)S == Y || (const void*)V == Y || U == S || U == V ||
      S == V)
    return fail(c, TSVD_EINVAL, "Y, U, S and V must be distinct buffers");
  if (!dims || order < 3 || order > 6) return fail(c, TSVD_EINVAL, "bad order or dims");
  for (int d = 0; d < order; ++d)
    if (dims[d] < 1) return fail(c, TSVD_EINVAL, "dims[%d] = %lld < 1", d, (long long)dims[d]);
  const int nv0 = (int)std::min(dims[0], dims[1]);
  if (k < 0 || k > nv0) return fail(c, TSVD_EINVAL, "k = %d outside [0, min(n1, n2) = %d]", k, nv0);
  if (k == 0) k = nv0;
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int ku = pointer_kind(U, c->device), ks = pointer_kind(S, c->device);
  const int kv = pointer_kind(V, c->device);
  if (ku < 0 || ks < 0 || kv < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  int64_t nsl = 1;
  for (int d = 2; d < order; ++d) nsl *= dims[d];
  const size_t nU = (size_t)dims[0] * k, nV = (size_t)dims[1] * k, nS = (size_t)k * k;
  int64_t nst = 1;   // stored Fourier slices, as make_problem counts them
  for (int d = 2; d < order - 1; ++d) nst *= dims[d];
  nst *= dims[order - 1] / 2 + 1;
  const size_t b_fu = align_up((size_t)nst * nU * sizeof(float2));
  const size_t b_fs = align_up((size_t)nst * nS * sizeof(float2));
  const size_t b_fv = align_up((size_t)nst * nV * sizeof(float2));
  const size_t b_ou = ku == 1 ? align_up((size_t)nsl * nU * sizeof(float)) : 0;
  const size_t b_os = ks == 1 ? align_up((size_t)nsl * nS * sizeof(float)) : 0;
  const size_t b_ov = kv == 1 ? align_up((size_t)nsl * nV * sizeof(float)) : 0;
  FactorWork fw;
  TSVD_TRY(factor_slices(c, Y, order, dims, b_fu + b_fs + b_fv + b_ou + b_os + b_ov, fw));
  char* b = fw.extra;
  float2* fU = reinterpret_cast<float2*>(b);
  float2* fS = reinterpret_cast<float2*>(b += b_fu);
  float2* fV = reinterpret_cast<float2*>(b += b_fs);
  b += b_fv;
  // outputs in host memory are written to staging first
  float* oU = U;
  float* oS = S;
  float* oV = V;
  if (ku == 1) {
    oU = reinterpret_cast<float*>(b);
    b += b_ou;
  }
  if (ks == 1) {
    oS = reinterpret_cast<float*>(b);
    b += b_os;
  }
  if (kv == 1) oV = reinterpret_cast<float*>(b);
  FactorArgs fa = factor_args(fw, k);
  fa.Uh = fU;
  fa.Sh = fS;
  fa.Vh = fV;
  TSVD_TRY(launch(c, launch_factor_assemble(fa, c->cur), "t-SVD factors"));
  // each factor is a tensor with the same tube geometry and its own tube count
  const struct {
    const float2* spec;
    float* out;
    size_t tubes;
  } outs[3] = {{fU, oU, nU}, {fS, oS, nS}, {fV, oV, nV}};
  for (const auto& o : outs) {
    TubeArgs t = tube_args(fw.p, fw.w, TUBE_INV);
    t.g.N12 = (int64_t)o.tubes;
    t.spec_in = o.spec;
    t.out0 = o.out;
    TSVD_TRY(run_tube(c, t, "tube pass (inverse)"));
  }
  if (ku == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(U, oU, nsl * nU * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (ks == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(S, oS, nsl * nS * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (kv == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(V, oV, nsl * nV * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  bool conv = true;
  TSVD_TRY(read_slice_stats(c, fw.p, fw.w, nullptr, nullptr, nullptr, &conv));
  if (!conv) return fail(c, TSVD_ENOTCONV, "a slice SVD reached max_sweeps = %d", c->opts.max_sweeps);
  return TSVD_OK;
}

// t-SVD compression (Sec. 3, Methods 1 and 2): the slice SVDs, the per-slice numbers of kept
// terms chosen here from the singular values, the slices rebuilt from their kept terms
// (factor.cu) and one inverse tube pass.
tsvd_status tsvd_compress(tsvd_ctx* c, const float* Y, int order, const int64_t* dims, int method,
                          int64_t k, float* Z, int64_t* kept_total, double* ratio) {
  if (!c) return TSVD_EINVAL;
  begin_call(c);
  if (!Y || !Z) return fail(c, TSVD_EINVAL, "Y and Z must not be NULL");
  if (method != TSVD_COMPRESS_GLOBAL && method != TSVD_COMPRESS_TUBAL)
    return fail(c, TSVD_EINVAL, "method must be TSVD_COMPRESS_GLOBAL or TSVD_COMPRESS_TUBAL");
  if (!dims || order < 3 || order > 6) return fail(c, TSVD_EINVAL, "bad order or dims");
  for (int d = 0; d < order; ++d)
    if (dims[d] < 1) return fail(c, TSVD_EINVAL, "dims[%d] = %lld < 1", d, (long long)dims[d]);
  int64_t nsl = 1;
  for (int d = 2; d < order; ++d) nsl *= dims[d];
  const int64_t n0 = std::min(dims[0], dims[1]);
  const int64_t kmax = method == TSVD_COMPRESS_GLOBAL ? n0 * nsl : n0;
  if (k < 1 || k > kmax)
    return fail(c, TSVD_EINVAL, "k = %lld outside [1, %lld]", (long long)k, (long long)kmax);
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int kz = pointer_kind(Z, c->device);
  if (kz < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  int64_t nst = 1;
  for (int d = 2; d < order - 1; ++d) nst *= dims[d];
  nst *= dims[order - 1] / 2 + 1;
  const size_t b_k = align_up((size_t)nst * sizeof(int));
  const size_t b_z = kz == 1 ? align_up((size_t)nsl * dims[0] * dims[1] * sizeof(float)) : 0;
  FactorWork fw;
  TSVD_TRY(factor_slices(c, Y, order, dims, b_k + b_z, fw));
  const TubeGeom& g = fw.p.g;
  const int nv = fw.nv;
  int* kept_dev = reinterpret_cast<int*>(fw.extra);
  float* z = kz == 1 ? reinterpret_cast<float*>(fw.extra + b_k) : Z;
  // singular values of the distinct slices -> kept terms per stored slice
  std::vector<float> sig((size_t)g.nstore * nv);
  TSVD_CUDA(c, cudaMemcpyAsync(sig.data(), fw.sig, sig.size() * sizeof(float),
                               cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int> kept((size_t)g.nstore, 0);
  int64_t total = 0;
  if (method == TSVD_COMPRESS_TUBAL) {
    // Method 2: the first k singular tubes, i.e. the k largest singular values of every slice
    std::fill(kept.begin(), kept.end(), (int)k);
    total = k;
  } else {
    // Method 1: the k largest f-diagonal entries of S-hat over all n0 * nslices of them (a
    // distinct stored slice stands for 1 or 2 full-spectrum slices); entries equal to the
    // k-th largest are all kept, so conjugate slices keep the same terms and Z stays real
    std::vector<std::pair<float, int>> all;
    all.reserve((size_t)fw.w.ndistinct * nv);
    for (int kh = 0; kh < g.hh; ++kh)
      for (int kf = 0; kf < g.nf; ++kf) {
        if (!slice_is_distinct(g, kf, kh)) continue;
        const int q = kf + g.nf * kh, wgt = slice_weight(g, kf, kh);
        for (int v = 0; v < nv; ++v) all.push_back({sig[(size_t)q * nv + v], wgt});
      }
    std::sort(all.begin(), all.end(),
              [](const std::pair<float, int>& a, const std::pair<float, int>& b) {
                return a.first > b.first;
              });
    int64_t acc = 0;
    float thr = 0.f;
    for (const auto& e : all) {
      acc += e.second;
      thr = e.first;
      if (acc >= k) break;
    }
    for (int kh = 0; kh < g.hh; ++kh)
      for (int kf = 0; kf < g.nf; ++kf) {
        if (!slice_is_distinct(g, kf, kh)) continue;
        const int q = kf + g.nf * kh;
        int cnt = 0;
        for (int v = 0; v < nv; ++v) cnt += sig[(size_t)q * nv + v] >= thr ? 1 : 0;
        kept[(size_t)q] = cnt;
        total += (int64_t)cnt * slice_weight(g, kf, kh);
      }
  }
  TSVD_CUDA(c, cudaMemcpyAsync(kept_dev, kept.data(), kept.size() * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  FactorArgs fa = factor_args(fw, 1);
  TSVD_TRY(launch(c, launch_compress_rebuild(fa, kept_dev, fw.w.spec_b, c->cur),
                  "compression rebuild"));
  TubeArgs inv = tube_args(fw.p, fw.w, TUBE_INV);
  inv.spec_in = fw.w.spec_b;
  inv.out0 = z;
  TSVD_TRY(run_tube(c, inv, "tube pass (inverse)"));
  if (kz == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(Z, z, (size_t)fw.p.N * sizeof(float), cudaMemcpyDeviceToHost,
                                 c->stream));
  bool conv = true;
  TSVD_TRY(read_slice_stats(c, fw.p, fw.w, nullptr, nullptr, nullptr, &conv));
  if (!conv) return fail(c, TSVD_ENOTCONV, "a slice SVD reached max_sweeps = %d", c->opts.max_sweeps);
  const double n1 = (double)dims[0], n2 = (double)dims[1];
  if (kept_total) *kept_total = total;
  if (ratio)
    *ratio = method == TSVD_COMPRESS_TUBAL ? n1 * n2 / ((double)total * (n1 + n2 + 1.0))
                                           : n1 * n2 * (double)nsl / ((double)total * (n1 + n2 + 1.0));
  return TSVD_OK;
}

// t-product C = A * B (Def. 2.1.1; for order > 3 the product of the Fourier slices over every
// mode from 3 on): forward tube passes of A and B, one complex product per stored Fourier
// slice, one inverse tube pass.  Slices on the self-conjugate columns whose partner has the
// smaller full index are computed too (the inverse pass reads their partners instead).
tsvd_status tsvd_tproduct(tsvd_ctx* c, const float* A, const float* B, float* C, int order,
                          const int64_t* dims, int64_t n4) {
  if (!c) return TSVD_EINVAL;
  begin_call(c);
  if (!A || !B || !C) return fail(c, TSVD_EINVAL, "A, B and C must not be NULL");
  if ((const void*)C == A || (const void*)C == B)
    return fail(c, TSVD_EINVAL, "C must not alias A or B");
  if (!dims || order < 3 || order > 6) return fail(c, TSVD_EINVAL, "bad order or dims");
  for (int d = 0; d < order; ++d)
    if (dims[d] < 1) return fail(c, TSVD_EINVAL, "dims[%d] = %lld < 1", d, (long long)dims[d]);
  if (n4 < 1 || n4 > (1 << 30)) return fail(c, TSVD_EINVAL, "n4 = %lld outside [1, 2^30]", (long long)n4);
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int ka = pointer_kind(A, c->device), kb = pointer_kind(B, c->device);
  const int kc = pointer_kind(C, c->device);
  if (ka < 0 || kb < 0 || kc < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  Problem p;   // the tube geometry of A (B and C share its modes 3..N)
  TSVD_TRY(make_problem(c, order, dims, p, false));
  const int64_t n1 = p.n1, n2 = p.n2, nsl = p.nslices, nst = p.g.nstore;
  if (std::max(n1, n2) * n4 > (INT64_MAX / 16) / nsl)
    return fail(c, TSVD_EUNSUPPORTED, "tensor too large");
  const size_t rA = (size_t)(n1 * n2), rB = (size_t)(n2 * n4), rC = (size_t)(n1 * n4);
  const size_t b_tw = align_up(twid_count(p.g) * sizeof(float2));
  const size_t b_fa = align_up((size_t)nst * rA * sizeof(float2));
  const size_t b_fb = align_up((size_t)nst * rB * sizeof(float2));
  const size_t b_fc = align_up((size_t)nst * rC * sizeof(float2));
  const size_t b_sa = ka == 1 ? align_up((size_t)nsl * rA * sizeof(float)) : 0;
  const size_t b_sb = kb == 1 ? align_up((size_t)nsl * rB * sizeof(float)) : 0;
  const size_t b_sc = kc == 1 ? align_up((size_t)nsl * rC * sizeof(float)) : 0;
  TSVD_TRY(grow_fbuf(c, b_tw + b_fa + b_fb + b_fc + b_sa + b_sb + b_sc));
  char* b = c->fbuf;
  Workspace w;
  w.twid = reinterpret_cast<float2*>(b);
  float2* fA = reinterpret_cast<float2*>(b += b_tw);
  float2* fB = reinterpret_cast<float2*>(b += b_fa);
  float2* fC = reinterpret_cast<float2*>(b += b_fb);
  b += b_fc;
  const float* a = A;
  const float* bb = B;
  float* out = C;
  if (ka == 1) {
    float* st = reinterpret_cast<float*>(b);
    b += b_sa;
    TSVD_CUDA(c, cudaMemcpyAsync(st, A, nsl * rA * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    a = st;
  }
  if (kb == 1) {
    float* st = reinterpret_cast<float*>(b);
    b += b_sb;
    TSVD_CUDA(c, cudaMemcpyAsync(st, B, nsl * rB * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    bb = st;
  }
  if (kc == 1) out = reinterpret_cast<float*>(b);
  fill_twiddles(p.g, c->twid_host);
  TSVD_CUDA(c, cudaMemcpyAsync(w.twid, c->twid_host.data(), c->twid_host.size() * sizeof(float2),
                               cudaMemcpyHostToDevice, c->stream));
  const struct {
    const float* in;
    float2* spec;
    size_t tubes;
  } ins[2] = {{a, fA, rA}, {bb, fB, rB}};
  for (const auto& x : ins) {
    TubeArgs t = tube_args(p, w, TUBE_FWD);
    t.g.N12 = (int64_t)x.tubes;
    t.in = x.in;
    t.spec_out = x.spec;
    TSVD_TRY(run_tube(c, t, "tube pass (forward)"));
  }
  // C-hat_s = A-hat_s B-hat_s for every stored slice s, in batches of at most 65535
  const int engine = c->opts.precision == TSVD_PRECISION_FP32 ? RSVT_GEMM_FP32 : rsvt_engine(c);
  for (int64_t s0 = 0; s0 < nst; s0 += 65535) {
    CGemm g;
    g.M = (int)n1;
    g.N = (int)n4;
    g.K = (int)n2;
    g.batch = (int)std::min<int64_t>(65535, nst - s0);
    g.a = CMat{fA + (size_t)s0 * rA, nullptr, (int64_t)rA, 1, n1, 0};
    g.b = CMat{fB + (size_t)s0 * rB, nullptr, (int64_t)rB, 1, n2, 0};
    g.c = CMat{fC + (size_t)s0 * rC, nullptr, (int64_t)rC, 1, n1, 0};
    TSVD_TRY(record_event(c, 0));
    TSVD_TRY(launch(c, launch_cgemm(g, engine, c->stream), "slice products"));
    TSVD_TRY(record_event(c, 0));
  }
  TubeArgs t = tube_args(p, w, TUBE_INV);
  t.g.N12 = (int64_t)rC;
  t.spec_in = fC;
  t.out0 = out;
  TSVD_TRY(run_tube(c, t, "tube pass (inverse)"));
  if (kc == 1)
    TSVD_CUDA(c, cudaMemcpyAsync(C, out, nsl * rC * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (ka == 1 || kb == 1 || kc == 1) TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  return TSVD_OK;
}

}  // extern "C"

namespace {

tsvd_status complete_impl(tsvd_ctx* c, const float* M_obs, const uint8_t* omega, int order,
                          const int64_t* dims, int iters, const tsvd_admm_state* init,
                          float* X_out, float* Z_out, float* Q_out, tsvd_stats* stats) {
  if (!c) return TSVD_EINVAL;
  NvtxRange nr("tnn_complete");
  begin_call(c);
  if (!M_obs || !omega || !X_out) return fail(c, TSVD_EINVAL, "M_obs, omega and X_out must not be NULL");
  if (iters < 0) return fail(c, TSVD_EINVAL, "iters must be >= 0");
  if (init && iters < 1) return fail(c, TSVD_EINVAL, "a resumed solve runs at least 1 iteration");
  if (init && init->rho > 0 && !std::isfinite(init->rho))
    return fail(c, TSVD_EINVAL, "init->rho must be finite");
  Problem p;
  TSVD_TRY(make_problem(c, order, dims, p));
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int km = pointer_kind(M_obs, c->device), ko = pointer_kind(omega, c->device);
  const int kx = pointer_kind(X_out, c->device);
  const int kzz = Z_out ? pointer_kind(Z_out, c->device) : 0;
  if (km < 0 || ko < 0 || kx < 0 || kzz < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  {
    const void* st_ptrs[3] = {init ? init->Z : nullptr, init ? init->Q : nullptr, Q_out};
    for (const void* q : st_ptrs)
      if (q && pointer_kind(q, c->device) != 0)
        return fail(c, TSVD_EINVAL, "the ADMM state and Q_out must be device memory");
  }
  WsRequest rq;
  rq.state = rq.yn = true;
  rq.stage_in = km == 1;
  rq.stage_om = ko == 1;
  rq.stage_out0 = kx == 1;
  rq.stage_out1 = (Z_out && kzz == 1) || (Q_out && !Z_out);   // Z for Q_out
  rq.rsvt = mixed_precision(c);
  rq.warm = !rq.rsvt && c->opts.warm_start != TSVD_WARM_OFF && iters >= 2 &&
            warm_plan_exists(c, p);
  // the plans (and the scratch sized for them) are those of the V form when warm
  c->vform_now = rq.warm;
  Workspace w;
  TSVD_TRY(prepare_workspace(c, p, rq, w));
  const size_t bytes = (size_t)p.N * sizeof(float);
  const float* m = M_obs;
  const uint8_t* om = omega;
  if (km == 1) {
    TSVD_CUDA(c, cudaMemcpyAsync(w.stage_in, M_obs, bytes, cudaMemcpyHostToDevice, c->stream));
    m = w.stage_in;
  }
  if (ko == 1) {
    TSVD_CUDA(c, cudaMemcpyAsync(w.stage_om, omega, (size_t)p.N, cudaMemcpyHostToDevice, c->stream));
    om = w.stage_om;
  }
  float* x = kx == 1 ? w.stage_out0 : X_out;
  float* z = Z_out ? (kzz == 1 ? w.stage_out1 : Z_out) : (Q_out ? w.stage_out1 : nullptr);

  TSVD_TRY(launch(c, launch_encode_observed(m, om, w.yn, p.N, w.bad, c->stream), "encode observed"));
  int bad = 0;
  TSVD_CUDA(c, cudaMemcpyAsync(&bad, w.bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, TSVD_EINVAL, "%d observed entries are not finite", bad);

  const double scale = threshold_scale(c, p);
  const double rho_start = init && init->rho > 0 ? init->rho : c->opts.rho0;
  double rho = rho_start;
  if (iters == 0) {
    TSVD_TRY(launch(c, launch_project_observed(m, om, x, p.N, c->stream), "project"));
    if (z) TSVD_CUDA(c, cudaMemsetAsync(z, 0, bytes, c->stream));
    if (Q_out) TSVD_CUDA(c, cudaMemsetAsync(Q_out, 0, bytes, c->stream));
  } else {
    const bool tuned = !c->opts.autotune || c->tuned.count(plan_key(c, p, w.ndistinct));
    const SliceKnobs kn = planned_knobs(c, p, w.ndistinct);
    const std::vector<int64_t> key = solver_key(c, 1, p, iters, {m, om, x, z}, kn);
    double last_ratio = 1.0;
    auto body = [&]() -> tsvd_status {
      double r = rho_start;
      RsvtLoop rl(c, p, w);
      if (w.rsvt) TSVD_TRY(rl.begin());
      TubeArgs t0 = tube_args(p, w, TUBE_COMPLETE);
      t0.in = w.yn;
      t0.state = w.state;
      t0.spec_out = w.spec_a;
      t0.write_out = iters == 1;
      t0.out0 = x;
      if (!init) {
        // iteration 0: X = P_Omega(M), Q = 0, V = X + Q
        t0.first = 1;
      } else {
        // resumed from (Z, Q): Z-hat = R2C(Z) and V = Z + Q, so the pass forms
        // Q = V - Z, X = P_Omega(M) + P_Omega^c(Z - Q) and V = X + Q as every later pass does
        if (init->Z) {
          TubeArgs f = tube_args(p, w, TUBE_FWD);
          f.in = init->Z;
          f.spec_out = w.spec_b;
          TSVD_TRY(run_tube(c, f, "tube pass (resumed Z)"));
        } else {
          TSVD_CUDA(c, cudaMemsetAsync(w.spec_b, 0, (size_t)p.g.nstore * p.g.N12 * sizeof(float2),
                                       c->cur));
        }
        TSVD_TRY(launch(c, launch_combine4(w.state, init->Z, 1.f, init->Q, 1.f, nullptr, 0.f,
                                           nullptr, 0.f, 1.f, p.N, c->cur),
                        "resumed state"));
        t0.first = 0;
        t0.spec_in = w.spec_b;
        t0.ratio = 1.f;
      }
      TSVD_TRY(run_tube(c, t0, "completion pass"));
      for (int k = 0; k < iters; ++k) {
        const float tau = (float)(scale / r);
        if (w.rsvt) {
          TSVD_TRY(rl.step(tau));
        } else {
          if (k == 0) TSVD_TRY(tune_slices(c, p, w, tau));
          TSVD_TRY(plain_slice_step(c, p, w, tau, k));
        }
        const double r_next = std::fmin(c->opts.mu * r, c->opts.rho_max);
        if (k + 1 < iters) {
          TubeArgs t = tube_args(p, w, TUBE_COMPLETE);
          t.in = w.yn;
          t.state = w.state;
          t.spec_in = w.spec_b;
          t.spec_out = w.spec_a;
          t.ratio = (float)(r / r_next);
          t.write_out = (k + 2 == iters);
          t.out0 = x;
          TSVD_TRY(run_tube(c, t, "completion pass"));
        }
        last_ratio = r / r_next;
        r = r_next;
      }
      if (z) {
        TubeArgs inv = tube_args(p, w, TUBE_INV);
        inv.spec_in = w.spec_b;
        inv.out0 = z;
        TSVD_TRY(run_tube(c, inv, "tube pass (inverse)"));
      }
      if (Q_out)   // the scaled dual of the last iteration: (V - Z) rho_{k} / rho_{k+1}
        TSVD_TRY(launch(c, launch_combine4(Q_out, w.state, 1.f, z, -1.f, nullptr, 0.f, nullptr,
                                           0.f, (float)last_ratio, p.N, c->cur),
                        "final dual"));
      if (w.rsvt) TSVD_TRY(rl.finish());
      return TSVD_OK;
    };
    TSVD_TRY(run_maybe_graph(c, key, tuned && !w.rsvt && !init && !Q_out, body));
    for (int k = 0; k < iters; ++k) rho = std::fmin(c->opts.mu * rho, c->opts.rho_max);
  }
  if (kx == 1) TSVD_CUDA(c, cudaMemcpyAsync(X_out, x, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (z && kzz == 1) TSVD_CUDA(c, cudaMemcpyAsync(Z_out, z, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (kx == 1 || (z && kzz == 1)) TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  TSVD_TRY(fill_stats(c, p, w, iters, rho, stats));
  TSVD_CUDA(c, cudaGetLastError());
  return TSVD_OK;
}

tsvd_status rpca_impl(tsvd_ctx* c, const float* M, int order, const int64_t* dims, float lambda,
                      int iters, const tsvd_admm_state* init, float* L_out, float* S_out,
                      float* W_out, tsvd_stats* stats) {
  if (!c) return TSVD_EINVAL;
  NvtxRange nr("trpca");
  begin_call(c);
  if (!M || !L_out || !S_out) return fail(c, TSVD_EINVAL, "M, L_out and S_out must not be NULL");
  if (iters < 0) return fail(c, TSVD_EINVAL, "iters must be >= 0");
  if (init && iters < 1) return fail(c, TSVD_EINVAL, "a resumed solve runs at least 1 iteration");
  if (init && init->rho > 0 && !std::isfinite(init->rho))
    return fail(c, TSVD_EINVAL, "init->rho must be finite");
  if (!(lambda > 0.f) || !std::isfinite(lambda)) return fail(c, TSVD_EINVAL, "lambda must be finite and > 0");
  Problem p;
  TSVD_TRY(make_problem(c, order, dims, p));
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  const int km = pointer_kind(M, c->device), kl = pointer_kind(L_out, c->device);
  const int ks = pointer_kind(S_out, c->device);
  if (km < 0 || kl < 0 || ks < 0) return fail(c, TSVD_EINVAL, "tensor on another device");
  {
    const void* st_ptrs[3] = {init ? init->S : nullptr, init ? init->W : nullptr, W_out};
    for (const void* q : st_ptrs)
      if (q && pointer_kind(q, c->device) != 0)
        return fail(c, TSVD_EINVAL, "the ADMM state and W_out must be device memory");
  }
  WsRequest rq;
  rq.state = true;
  rq.stage_in = km == 1;
  rq.stage_out0 = kl == 1;
  rq.stage_out1 = ks == 1;
  rq.rsvt = mixed_precision(c);
  rq.warm = !rq.rsvt && c->opts.warm_start != TSVD_WARM_OFF && iters >= 2 &&
            warm_plan_exists(c, p);
  // the plans (and the scratch sized for them) are those of the V form when warm
  c->vform_now = rq.warm;
  Workspace w;
  TSVD_TRY(prepare_workspace(c, p, rq, w));
  const size_t bytes = (size_t)p.N * sizeof(float);
  const float* m = M;
  if (km == 1) {
    TSVD_CUDA(c, cudaMemcpyAsync(w.stage_in, M, bytes, cudaMemcpyHostToDevice, c->stream));
    m = w.stage_in;
  }
  float* l = kl == 1 ? w.stage_out0 : L_out;
  float* sp = ks == 1 ? w.stage_out1 : S_out;
  TSVD_TRY(launch(c, launch_count_nonfinite(m, p.N, w.bad, c->stream), "check input"));
  int bad = 0;
  TSVD_CUDA(c, cudaMemcpyAsync(&bad, w.bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, TSVD_EINVAL, "%d entries of M are not finite", bad);

  const double scale = threshold_scale(c, p);
  const double rho_start = init && init->rho > 0 ? init->rho : c->opts.rho0;
  double rho = rho_start;
  if (iters == 0) {
    TSVD_CUDA(c, cudaMemsetAsync(l, 0, bytes, c->stream));
    TSVD_CUDA(c, cudaMemsetAsync(sp, 0, bytes, c->stream));
    if (W_out) TSVD_CUDA(c, cudaMemsetAsync(W_out, 0, bytes, c->stream));
  } else {
    const bool tuned = !c->opts.autotune || c->tuned.count(plan_key(c, p, w.ndistinct));
    const SliceKnobs kn = planned_knobs(c, p, w.ndistinct);
    std::vector<int64_t> key = solver_key(c, 2, p, iters, {m, l, sp}, kn);
    int64_t lbits;
    std::memcpy(&lbits, &lambda, sizeof lambda);
    key.push_back(lbits);
    double last_ratio = 1.0;
    auto body = [&]() -> tsvd_status {
      double r = rho_start;
      RsvtLoop rl(c, p, w);
      if (w.rsvt) TSVD_TRY(rl.begin());
      TubeArgs t0 = tube_args(p, w, TUBE_FWD);
      t0.spec_out = w.spec_a;
      if (!init) {
        // iteration 0: S = W = 0, so the t-SVT input is M itself
        t0.in = m;
      } else {
        // resumed from (S, W): the t-SVT input M - S - W (staged in the output spectrum's
        // buffer, which the first slice SVT writes only after this pass), and W in the state
        float* v0 = reinterpret_cast<float*>(w.spec_b);
        TSVD_TRY(launch(c, launch_combine4(v0, m, 1.f, init->S, -1.f, init->W, -1.f, nullptr,
                                           0.f, 1.f, p.N, c->cur),
                        "resumed input"));
        TSVD_TRY(launch(c, launch_combine4(w.state, init->W, 1.f, nullptr, 0.f, nullptr, 0.f,
                                           nullptr, 0.f, 1.f, p.N, c->cur),
                        "resumed state"));
        t0.in = v0;
      }
      TSVD_TRY(run_tube(c, t0, "tube pass (forward)"));
      for (int k = 0; k < iters; ++k) {
        const float tau = (float)(scale / r);
        if (w.rsvt) {
          TSVD_TRY(rl.step(tau));
        } else {
          if (k == 0) TSVD_TRY(tune_slices(c, p, w, tau));
          TSVD_TRY(plain_slice_step(c, p, w, tau, k));
        }
        const double r_next = std::fmin(c->opts.mu * r, c->opts.rho_max);
        TubeArgs t = tube_args(p, w, TUBE_RPCA);
        t.in = m;
        t.state = w.state;
        t.spec_in = w.spec_b;
        t.spec_out = w.spec_a;
        t.ratio = (float)(r / r_next);
        t.kappa = (float)((double)lambda / r);
        t.first = k == 0 && !init;
        t.last = k + 1 == iters;
        t.out0 = l;
        t.out1 = sp;
        t.tube_sparse = c->opts.sparse_mode == TSVD_SPARSE_TUBE;
        TSVD_TRY(run_tube(c, t, "RPCA pass"));
        last_ratio = r / r_next;
        r = r_next;
      }
      // the scaled dual of the last iteration, (W + L + S - M) rho_k / rho_{k+1} (the last
      // pass writes L and S and leaves W as it was)
      if (W_out)
        TSVD_TRY(launch(c, launch_combine4(W_out, w.state, 1.f, l, 1.f, sp, 1.f, m, -1.f,
                                           (float)last_ratio, p.N, c->cur),
                        "final dual"));
      if (w.rsvt) TSVD_TRY(rl.finish());
      return TSVD_OK;
    };
    TSVD_TRY(run_maybe_graph(c, key, tuned && !w.rsvt && !init && !W_out, body));
    for (int k = 0; k < iters; ++k) rho = std::fmin(c->opts.mu * rho, c->opts.rho_max);
  }
  if (kl == 1) TSVD_CUDA(c, cudaMemcpyAsync(L_out, l, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (ks == 1) TSVD_CUDA(c, cudaMemcpyAsync(S_out, sp, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (kl == 1 || ks == 1) TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  TSVD_TRY(fill_stats(c, p, w, iters, rho, stats));
  TSVD_CUDA(c, cudaGetLastError());
  return TSVD_OK;
}

}  // namespace

extern "C" {

tsvd_status tnn_complete(tsvd_ctx* c, const float* M_obs, const uint8_t* omega, int order,
                         const int64_t* dims, int iters, float* X_out, float* Z_out,
                         tsvd_stats* stats) {
  return complete_impl(c, M_obs, omega, order, dims, iters, nullptr, X_out, Z_out, nullptr, stats);
}

tsvd_status tnn_complete_resume(tsvd_ctx* c, const float* M_obs, const uint8_t* omega, int order,
                                const int64_t* dims, int iters, const tsvd_admm_state* init,
                                float* X_out, float* Z_out, float* Q_out, tsvd_stats* stats) {
  return complete_impl(c, M_obs, omega, order, dims, iters, init, X_out, Z_out, Q_out, stats);
}

tsvd_status trpca(tsvd_ctx* c, const float* M, int order, const int64_t* dims, float lambda,
                  int iters, float* L_out, float* S_out, tsvd_stats* stats) {
  return rpca_impl(c, M, order, dims, lambda, iters, nullptr, L_out, S_out, nullptr, stats);
}

tsvd_status trpca_resume(tsvd_ctx* c, const float* M, int order, const int64_t* dims,
                         float lambda, int iters, const tsvd_admm_state* init, float* L_out,
                         float* S_out, float* W_out, tsvd_stats* stats) {
  return rpca_impl(c, M, order, dims, lambda, iters, init, L_out, S_out, W_out, stats);
}

}  // extern "C"

namespace {

// ---- persistent batched solves (plain form)
BatchTensor batch_tensor(tsvd_ctx* c, const BatchItem& it) {
  BatchTensor t{};
  const tsvd_problem& q = *it.src;
  t.g = it.p.g;
  t.kind = q.kind;
  t.n1 = (int)it.p.n1;
  t.n2 = (int)it.p.n2;
  t.nslices = it.w.ndistinct;
  t.warm = it.warm ? 1 : 0;
  t.scale = threshold_scale(c, it.p);
  t.lambda = q.lambda;
  t.tube_sparse = c->opts.sparse_mode == TSVD_SPARSE_TUBE;
  t.spec_a = it.w.spec_a;
  t.spec_b = it.w.spec_b;
  t.state = it.w.state;
  t.in = q.kind == TSVD_PROBLEM_COMPLETE ? it.w.yn : q.M;
  t.twid_h = it.w.twid;
  t.twid_f = it.w.twid ? it.w.twid + it.p.g.nh : nullptr;
  t.slices = it.w.slices;
  t.stat = it.w.stat;
  t.acc = it.w.acc;
  t.vwarm = it.w.vwarm;
  t.out0 = q.out0;
  t.out1 = q.out1;
  return t;
}

// Plans a persistent batched solve may use: (cluster size, single-CTA threshold), the
// threshold 2 C x 16 (blocks of at least 16 vectors) or none (single-CTA slices only where a
// cluster plan does not fit).
std::vector<std::array<int, 2>> batch_candidates() {
  std::vector<std::array<int, 2>> out;
  for (int C : {2, 4, 8}) {
    out.push_back({C, 2 * C * 16});
    out.push_back({C, 0});
  }
  return out;
}

std::vector<int64_t> batch_signature(const std::vector<BatchItem>& items) {
  std::vector<int64_t> key;
  for (const BatchItem& it : items) {
    const int64_t v[] = {it.src->kind, it.p.n1, it.p.n2, it.p.g.nf, it.p.g.nh, it.warm ? 1 : 0};
    key.insert(key.end(), std::begin(v), std::end(v));
  }
  return key;
}

// The persistent batched solve: tensors' regions carved and initialised, inputs checked.
// ctr: 3 (iters + 1) queue counters, then one completion counter per tensor, then the error
// word.  On the first call with a new batch shape every candidate plan is timed on iteration
// 0's slice SVTs (sweeps capped at 4) and the fastest kept; then the init launch and one
// launch per iteration run (captured into a graph with use_graphs), and the call waits for
// the error word.
tsvd_status persistent_batch(tsvd_ctx* c, const std::vector<BatchItem>& items, int iters,
                             const std::vector<std::array<int, 2>>& cands, char* table_dev,
                             char* scratch, int* ctr) {
  const int count = (int)items.size();
  unsigned* done = reinterpret_cast<unsigned*>(ctr + 3 * (iters + 1));
  int* err = reinterpret_cast<int*>(done + count);
  std::vector<BatchTensor> ts;
  for (const BatchItem& it : items) ts.push_back(batch_tensor(c, it));
  BatchPlan plan;
  auto make = [&](const std::array<int, 2>& cd) -> tsvd_status {
    if (!batch_plan(ts.data(), count, cd[0], cd[1], plan, c->batch_table))
      return fail(c, TSVD_EUNSUPPORTED, "no persistent batch plan");
    TSVD_CUDA(c, cudaMemcpyAsync(table_dev, c->batch_table.data(), plan.table_bytes,
                                 cudaMemcpyHostToDevice, c->cur));
    return TSVD_OK;
  };
  auto reset = [&]() -> tsvd_status {
    TSVD_CUDA(c, cudaMemsetAsync(ctr, 0,
                                 3 * ((size_t)iters + 1) * sizeof(int) + (size_t)count * sizeof(unsigned) +
                                     sizeof(int),
                                 c->cur));
    return TSVD_OK;
  };
  BatchIter bi{};
  bi.iters = iters;
  bi.tol = c->opts.jacobi_tol;
  bi.max_sweeps = c->opts.max_sweeps;
  bi.abs_stop = c->opts.jacobi_stop == TSVD_STOP_SVT ? 1 : 0;
  bi.done = done;
  bi.err = err;
  auto run = [&](int k, double r, double r_next, bool slices_only) -> tsvd_status {
    NvtxRange nr("persistent batched iteration");
    bi.k = k;
    bi.r = r;
    bi.r_next = r_next;
    bi.ctr = ctr + 3 * (k + 1);
    bi.slices_only = slices_only ? 1 : 0;
    TSVD_TRY(record_event(c, 0));
    TSVD_TRY(launch(c, launch_batch_iteration(plan, table_dev, scratch, bi, c->cur),
                    "persistent batched iteration"));
    if (k >= 0) ++c->slice_launches;
    return record_event(c, 0);
  };
  const std::vector<int64_t> sig = batch_signature(items);
  auto tuned = c->batch_tuned.find(sig);
  if (tuned == c->batch_tuned.end()) {
    std::array<int, 2> best = cands[0];
    if (cands.size() > 1 && c->opts.autotune) {
      // time iteration 0's slice SVTs of every candidate on the real first spectra
      c->cur = c->stream;
      TSVD_TRY(make(cands[0]));
      TSVD_TRY(reset());
      TSVD_TRY(run(-1, c->opts.rho0, c->opts.rho0, false));
      cudaEvent_t e0, e1;
      TSVD_CUDA(c, cudaEventCreate(&e0));
      if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, TSVD_ECUDA, "cudaEventCreate failed");
      }
      const int ms_keep = bi.max_sweeps;
      bi.max_sweeps = std::min(4, ms_keep);
      float best_ms = 1e30f;
      tsvd_status st = TSVD_OK;
      for (const auto& cd : cands) {
        if ((st = make(cd)) != TSVD_OK) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == TSVD_OK; ++rep) {   // the first run loads the kernel
          // iteration 0's queue counters and the completion counters start from zero
          TSVD_CUDA(c, cudaMemsetAsync(ctr + 3, 0, 3 * sizeof(int), c->cur));
          TSVD_CUDA(c, cudaMemsetAsync(done, 0, (size_t)count * sizeof(unsigned), c->cur));
          cudaEventRecord(e0, c->cur);
          st = run(0, c->opts.rho0, c->opts.rho0, true);
          cudaEventRecord(e1, c->cur);
        }
        if (st != TSVD_OK) break;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best_ms) {
          best_ms = ms;
          best = cd;
        }
      }
      bi.max_sweeps = ms_keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (st != TSVD_OK) return st;
      TSVD_CUDA(c, cudaGetLastError());
      // the timing runs added to the per-tensor counters
      for (const BatchItem& it : items) {
        TSVD_CUDA(c, cudaMemsetAsync(it.w.acc, 0, sizeof(SweepAccum), c->cur));
        TSVD_CUDA(c, cudaMemsetAsync(it.w.stat, 0, (size_t)it.p.g.nstore * sizeof(SliceStat), c->cur));
      }
      c->launches = 0;
      c->slice_launches = 0;
      c->events_used = 0;
    }
    tuned = c->batch_tuned.emplace(sig, best).first;
  }
  c->cur = c->stream;
  TSVD_TRY(make(tuned->second));
  std::vector<int64_t> key = {4, count, iters, (int64_t)(intptr_t)c->ws, (int64_t)c->ws_cap,
                              c->opts.tnn_scale, c->opts.sparse_mode, c->opts.max_sweeps,
                              c->opts.timing, tuned->second[0], tuned->second[1]};
  double d[4] = {c->opts.rho0, c->opts.mu, c->opts.rho_max, (double)c->opts.jacobi_tol};
  for (double v : d) {
    int64_t bits;
    std::memcpy(&bits, &v, sizeof bits);
    key.push_back(bits);
  }
  for (const BatchItem& it : items) {
    const tsvd_problem& q = *it.src;
    int64_t lbits = 0;
    std::memcpy(&lbits, &q.lambda, sizeof q.lambda);
    const int64_t vals[] = {q.kind, q.order, q.dims[0], q.dims[1], q.dims[2],
                            q.order == 4 ? q.dims[3] : 1, (int64_t)(intptr_t)q.M,
                            (int64_t)(intptr_t)q.omega, (int64_t)(intptr_t)q.out0,
                            (int64_t)(intptr_t)q.out1, lbits, it.warm ? 1 : 0};
    key.insert(key.end(), std::begin(vals), std::end(vals));
  }
  auto body = [&]() -> tsvd_status {
    TSVD_TRY(reset());
    double r = c->opts.rho0;
    TSVD_TRY(run(-1, r, r, false));
    for (int k = 0; k < iters; ++k) {
      const double r_next = std::fmin(c->opts.mu * r, c->opts.rho_max);
      TSVD_TRY(run(k, r, r_next, false));
      r = r_next;
    }
    return TSVD_OK;
  };
  TSVD_TRY(run_maybe_graph(c, key, true, body));
  int err_h = 0;
  TSVD_CUDA(c, cudaMemcpyAsync(&err_h, err, sizeof err_h, cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  if (err_h) return fail(c, TSVD_ETIMEOUT, "a persistent batched launch gave up a bounded wait");
  return TSVD_OK;
}

// The batched solve behind tsvd_solve_batched (only_kind = 0: any mix of problems) and
// tnn_complete_batched / trpca_batched (every problem must be of kind only_kind).
tsvd_status solve_batched(tsvd_ctx* c, int count, const tsvd_problem* problems, int iters,
                          tsvd_stats* stats, int only_kind) {
  if (!c) return TSVD_EINVAL;
  NvtxRange nr("batched solve");
  begin_call(c);
  if (count < 0 || (count > 0 && !problems)) return fail(c, TSVD_EINVAL, "bad problem list");
  if (only_kind)
    for (int i = 0; i < count; ++i)
      if (problems[i].kind != only_kind)
        return fail(c, TSVD_EINVAL, "problem %d: kind %d in a %s call", i, problems[i].kind,
                    only_kind == TSVD_PROBLEM_COMPLETE ? "tnn_complete_batched"
                                                       : "trpca_batched");
  if (iters < 0) return fail(c, TSVD_EINVAL, "iters must be >= 0");
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  std::vector<BatchItem> items((size_t)count);
  for (int i = 0; i < count; ++i) {
    const tsvd_problem& q = problems[i];
    BatchItem& it = items[(size_t)i];
    it.src = &q;
    if (q.kind != TSVD_PROBLEM_COMPLETE && q.kind != TSVD_PROBLEM_RPCA)
      return fail(c, TSVD_EINVAL, "problem %d: bad kind %d", i, q.kind);
    if (q.order != 3 && q.order != 4)
      return fail(c, TSVD_EINVAL, "problem %d: batched tensors are 3-way or 4-way", i);
    tsvd_status st = make_problem(c, q.order, q.dims, it.p);
    if (st != TSVD_OK) return fail(c, st, "problem %d: %s", i, c->err.c_str());
    const bool complete = q.kind == TSVD_PROBLEM_COMPLETE;
    if (!q.M || !q.out0 || (complete && !q.omega) || (!complete && !q.out1))
      return fail(c, TSVD_EINVAL, "problem %d: missing buffer", i);
    if (!complete && (!(q.lambda > 0.f) || !std::isfinite(q.lambda)))
      return fail(c, TSVD_EINVAL, "problem %d: lambda must be finite and > 0", i);
    const void* ptrs[4] = {q.M, complete ? (const void*)q.omega : nullptr, q.out0, q.out1};
    for (const void* ptr : ptrs)
      if (ptr && pointer_kind(ptr, c->device) != 0)
        return fail(c, TSVD_EINVAL, "problem %d: batched tensors must be device memory", i);
  }
  if (count == 0) {
    if (stats) std::memset(stats, 0, sizeof *stats);
    return TSVD_OK;
  }
  // the plain form runs as one persistent launch per iteration when every tensor has a plan
  bool persist = !mixed_precision(c) && c->opts.batch_persistent && iters > 0;
  std::vector<std::array<int, 2>> cands;
  size_t table_cap = 0, scratch_cap = 0;
  if (persist) {
    for (BatchItem& it : items) carve_item(c, it, nullptr, iters, true);
    std::vector<BatchTensor> ts;
    for (const BatchItem& it : items) ts.push_back(batch_tensor(c, it));
    for (const auto& cd : batch_candidates()) {
      BatchPlan pl;
      std::vector<unsigned char> tab;
      if (!batch_plan(ts.data(), count, cd[0], cd[1], pl, tab)) continue;
      cands.push_back(cd);
      table_cap = std::max(table_cap, pl.table_bytes);
      scratch_cap = std::max(scratch_cap, pl.scratch_bytes);
    }
    persist = !cands.empty();
  }
  // one allocation for every tensor's regions plus the batch's non-finite counters (and for
  // the persistent launch its table, exchange buffers, queue counters and error word)
  size_t total = 0;
  std::vector<size_t> offs((size_t)count);
  for (int i = 0; i < count; ++i) {
    offs[(size_t)i] = total;
    total += carve_item(c, items[(size_t)i], nullptr, iters, persist);
  }
  // a forced slice plan (ctas_per_slice, lanes_per_pair) that some tensor's slices do not fit
  // is refused here, before anything is enqueued on the branches
  if (!mixed_precision(c) && !persist && iters > 0)
    for (int i = 0; i < count; ++i) {
      const BatchItem& it = items[(size_t)i];
      if (!jacobi_svt_plan_ok((int)it.p.n1, (int)it.p.n2, it.w.ndistinct, it.kn))
        return fail(c, TSVD_EUNSUPPORTED,
                    "problem %d: no slice SVT plan for %lld x %lld slices with %d CTAs per slice "
                    "and %d lanes per pair",
                    i, (long long)it.p.n1, (long long)it.p.n2, it.kn.ctas, it.kn.lanes);
    }
  const size_t bad_off = total;
  total += align_up((size_t)count * sizeof(int));
  const size_t table_off = total;
  total += align_up(table_cap);
  const size_t scratch_off = total;
  total += align_up(scratch_cap);
  const size_t ctr_off = total;
  const size_t nctr = persist ? 3 * ((size_t)iters + 1) : 0;
  total += align_up(nctr * sizeof(int) + (size_t)count * sizeof(unsigned) + sizeof(int));
  if (total > c->ws_cap) {
    if (c->ws) {
      TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
      cudaFree(c->ws);
      c->ws = nullptr;
      c->ws_cap = 0;
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
      c->graphs.clear();
    }
    void* ptr = nullptr;
    cudaError_t e = device_alloc(&ptr, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, TSVD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", total, cudaGetErrorString(e));
    }
    c->ws = static_cast<char*>(ptr);
    c->ws_cap = total;
  }
  int* bad = reinterpret_cast<int*>(c->ws + bad_off);
  TSVD_CUDA(c, cudaMemsetAsync(bad, 0, (size_t)count * sizeof(int), c->stream));
  for (int i = 0; i < count; ++i) {
    BatchItem& it = items[(size_t)i];
    carve_item(c, it, c->ws + offs[(size_t)i], iters, persist);
    const TubeGeom& g = it.p.g;
    fill_twiddles(g, it.twid);   // same FP64 tables as the single-tensor calls
    TSVD_CUDA(c, cudaMemcpyAsync(it.w.twid, it.twid.data(), it.twid.size() * sizeof(float2),
                                 cudaMemcpyHostToDevice, c->stream));
    TSVD_CUDA(c, cudaMemcpyAsync(it.w.slices, it.slices.data(), it.slices.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, c->stream));
    TSVD_CUDA(c, cudaMemsetAsync(it.w.acc, 0, sizeof(SweepAccum), c->stream));
    TSVD_CUDA(c, cudaMemsetAsync(it.w.stat, 0, (size_t)g.nstore * sizeof(SliceStat), c->stream));
    if (it.w.rsvt)
      TSVD_CUDA(c, cudaMemcpyAsync(it.w.risreal, it.isreal.data(), it.isreal.size(),
                                   cudaMemcpyHostToDevice, c->stream));
    const tsvd_problem& q = *it.src;
    if (q.kind == TSVD_PROBLEM_COMPLETE)
      TSVD_TRY(launch(c, launch_encode_observed(q.M, q.omega, it.w.yn, it.p.N, bad + i, c->stream),
                      "encode observed"));
    else
      TSVD_TRY(launch(c, launch_count_nonfinite(q.M, it.p.N, bad + i, c->stream), "check input"));
  }
  std::vector<int> bad_h((size_t)count);
  TSVD_CUDA(c, cudaMemcpyAsync(bad_h.data(), bad, (size_t)count * sizeof(int),
                               cudaMemcpyDeviceToHost, c->stream));
  TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < count; ++i)
    if (bad_h[(size_t)i]) return fail(c, TSVD_EINVAL, "problem %d: %d entries are not finite", i, bad_h[(size_t)i]);

  double rho = c->opts.rho0;
  for (int k = 0; k < iters; ++k) rho = std::fmin(c->opts.mu * rho, c->opts.rho_max);
  if (iters == 0) {
    for (const BatchItem& it : items) {
      const tsvd_problem& q = *it.src;
      const size_t bytes = (size_t)it.p.N * sizeof(float);
      if (q.kind == TSVD_PROBLEM_COMPLETE) {
        TSVD_TRY(launch(c, launch_project_observed(q.M, q.omega, q.out0, it.p.N, c->stream), "project"));
        if (q.out1) TSVD_CUDA(c, cudaMemsetAsync(q.out1, 0, bytes, c->stream));
      } else {
        TSVD_CUDA(c, cudaMemsetAsync(q.out0, 0, bytes, c->stream));
        TSVD_CUDA(c, cudaMemsetAsync(q.out1, 0, bytes, c->stream));
      }
    }
  } else if (persist) {
    TSVD_TRY(persistent_batch(c, items, iters, cands, c->ws + table_off,
                              scratch_cap ? c->ws + scratch_off : nullptr,
                              reinterpret_cast<int*>(c->ws + ctr_off)));
  } else {
    // stream branches: every branch forks from and joins the issuing stream, so the tensors'
    // chains overlap on the GPU; up to 64 (one per tensor on the 64-tensor batch: the mixed
    // form's chains of small kernels gained 17% over 16 branches, the plain form 1%)
    const int nbr = std::min(count, 64);
    while ((int)c->branches.size() < nbr) {
      cudaStream_t s;
      cudaEvent_t e;
      TSVD_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      TSVD_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->branches.push_back(s);
      c->joins.push_back(e);
    }
    if (!c->fork) TSVD_CUDA(c, cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    std::vector<int64_t> key = {3, count, iters, (int64_t)(intptr_t)c->ws, (int64_t)c->ws_cap,
                                c->opts.tnn_scale, c->opts.sparse_mode, c->opts.max_sweeps,
                                c->opts.timing, c->opts.precision, c->opts.rsvt_oversample,
                                c->opts.rsvt_kmax};
    double d[4] = {c->opts.rho0, c->opts.mu, c->opts.rho_max, (double)c->opts.jacobi_tol};
    for (double v : d) {
      int64_t bits;
      std::memcpy(&bits, &v, sizeof bits);
      key.push_back(bits);
    }
    for (const BatchItem& it : items) {
      const tsvd_problem& q = *it.src;
      int64_t lbits = 0;
      std::memcpy(&lbits, &q.lambda, sizeof q.lambda);
      const int64_t vals[] = {q.kind, q.order, q.dims[0], q.dims[1], q.dims[2],
                              q.order == 4 ? q.dims[3] : 1, (int64_t)(intptr_t)q.M,
                              (int64_t)(intptr_t)q.omega, (int64_t)(intptr_t)q.out0,
                              (int64_t)(intptr_t)q.out1, lbits, it.kn.ctas, it.kn.lanes,
                              it.kn.ppg, it.kn.vform, it.warm ? 1 : 0};
      key.insert(key.end(), std::begin(vals), std::end(vals));
    }
    // tensors to branches by longest processing time first, on the estimated slice-SVT work
    // of a solve: m n^2 per distinct slice per sweep, ~3x fewer sweeps when warm-started
    std::vector<int> branch_of((size_t)count, 0), order((size_t)count);
    {
      std::vector<double> cost((size_t)count), load((size_t)nbr, 0.0);
      for (int i = 0; i < count; ++i) {
        const BatchItem& it = items[(size_t)i];
        const double m = (double)std::max(it.p.n1, it.p.n2), n = (double)std::min(it.p.n1, it.p.n2);
        cost[(size_t)i] = m * n * n * it.w.ndistinct * (it.warm ? 1.0 : 3.0) + m * n;
        order[(size_t)i] = i;
      }
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int b) { return cost[(size_t)a] > cost[(size_t)b]; });
      for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch_of[(size_t)i] = b;
        load[(size_t)b] += cost[(size_t)i];
      }
    }
    auto body = [&]() -> tsvd_status {
      cudaStream_t base = c->cur;
      TSVD_CUDA(c, cudaEventRecord(c->fork, base));
      for (int b = 0; b < nbr; ++b) TSVD_CUDA(c, cudaStreamWaitEvent(c->branches[(size_t)b], c->fork, 0));
      // the costliest tensors are issued first on their branches
      tsvd_status st = TSVD_OK;
      for (int i : order) {
        c->cur = c->branches[(size_t)branch_of[(size_t)i]];
        st = enqueue_item(c, items[(size_t)i], iters);
        if (st != TSVD_OK) break;
      }
      c->cur = base;
      // every branch joins the issuing stream even after a failed enqueue, so that no work
      // is left outside the stream order (or unjoined in a capture)
      for (int b = 0; b < nbr; ++b) {
        const cudaError_t e1 = cudaEventRecord(c->joins[(size_t)b], c->branches[(size_t)b]);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(base, c->joins[(size_t)b], 0) : e1;
        if (e2 != cudaSuccess && st == TSVD_OK)
          st = fail(c, TSVD_ECUDA, "branch join: %s", cudaGetErrorString(e2));
      }
      return st;
    };
    TSVD_TRY(run_maybe_graph(c, key, true, body));
  }
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    stats->iters = iters;
    stats->rho_final = rho;
    stats->launches = c->launches;
    stats->slice_launches = c->slice_launches;
    TSVD_TRY(timed_totals(c, &stats->slice_ms, &stats->tube_ms));
    if (iters > 0) {
      for (const BatchItem& it : items) {
        SweepAccum acc;
        TSVD_CUDA(c, cudaMemcpyAsync(&acc, it.w.acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
        int rmax = 0;
        double tnn = 0;
        TSVD_TRY(read_slice_stats(c, it.p, it.w, nullptr, &tnn, &rmax, nullptr));
        stats->max_sweeps_used = std::max(stats->max_sweeps_used, acc.max_sweeps);
        stats->total_sweeps += (int64_t)acc.total_sweeps;
        stats->nonconverged += (int64_t)acc.nonconverged;
        stats->slice_svds += (int64_t)iters * it.w.ndistinct;
        stats->tnn_last += tnn;
        stats->rank_last_max = std::max(stats->rank_last_max, rmax);
        if (it.w.rsvt) {
          RsvtStat rs;
          TSVD_CUDA(c, cudaMemcpyAsync(&rs, it.w.rstat, sizeof rs, cudaMemcpyDeviceToHost,
                                       c->stream));
          TSVD_CUDA(c, cudaStreamSynchronize(c->stream));
          stats->rsvt_k_last = std::max(stats->rsvt_k_last, rs.k);
          stats->rsvt_saturated += rs.saturated;
          stats->rsvt_drops += rs.drops;
          // algorithmic work of the iterations run, from the device-chosen widths: the three
          // complex products and the GvL count of the small SVDs (as the single-tensor calls)
          const double mw = it.w.mw, nw = it.w.nw, ns = it.w.ndistinct;
          stats->rsvt_gemm_gflop += ns * 3.0 * 8.0 * mw * nw * rs.ksum[0] * 1e-9;
          stats->rsvt_svd_gflop += ns * 4.0 * (4.0 * nw * rs.ksum[1] + 8.0 * rs.ksum[2]) * 1e-9;
        }
      }
    }
  }
  TSVD_CUDA(c, cudaGetLastError());
  return TSVD_OK;
}

}  // namespace

extern "C" {

tsvd_status tsvd_solve_batched(tsvd_ctx* c, int count, const tsvd_problem* problems, int iters,
                               tsvd_stats* stats) {
  return solve_batched(c, count, problems, iters, stats, 0);
}

tsvd_status tsvd_selftest_bounded_wait(int device, int limit_ms) {
  if (limit_ms < 0 || limit_ms > 10000) return TSVD_EINVAL;
  DeviceGuard dg(device);
  if (!dg.ok) {
    cudaGetLastError();
    return TSVD_ECUDA;
  }
  void* buf = nullptr;
  if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ENOMEM;
  }
  int err_h = 0;
  cudaError_t e = cudaMemset(buf, 0, 2 * sizeof(int));
  unsigned* counter = static_cast<unsigned*>(buf);
  int* err = static_cast<int*>(buf) + 1;
  if (e == cudaSuccess)
    e = launch_wait_selftest(counter, (unsigned long long)limit_ms * 1000000ull, err, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&err_h, err, sizeof err_h, cudaMemcpyDeviceToHost);
  cudaGetLastError();
  cudaFree(buf);
  if (e != cudaSuccess) return TSVD_ECUDA;
  return err_h ? TSVD_ETIMEOUT : TSVD_OK;
}

long long tsvd_fault_injection_reset(const char* spec) {
  g_fault_alloc_at = parse_fault_spec(spec ? spec : std::getenv("TSVD_FAULT"));
  g_alloc_count = 0;
  return g_fault_alloc_at.load();
}

tsvd_status tnn_complete_batched(tsvd_ctx* c, int count, const tsvd_problem* problems, int iters,
                                 tsvd_stats* stats) {
  return solve_batched(c, count, problems, iters, stats, TSVD_PROBLEM_COMPLETE);
}

tsvd_status trpca_batched(tsvd_ctx* c, int count, const tsvd_problem* problems, int iters,
                          tsvd_stats* stats) {
  return solve_batched(c, count, problems, iters, stats, TSVD_PROBLEM_RPCA);
}

tsvd_status tsvd_cgemm(tsvd_ctx* c, int transa, int transb, int m, int n, int k,
                       const float* A, int64_t lda, int64_t stride_a, const float* B,
                       int64_t ldb, int64_t stride_b, float* C, int64_t ldc, int64_t stride_c,
                       int batch) {
  if (!c) return TSVD_EINVAL;
  begin_call(c);
  auto op_ok = [](int t) { return t == TSVD_OP_N || t == TSVD_OP_T || t == TSVD_OP_C; };
  if (!op_ok(transa) || !op_ok(transb)) return fail(c, TSVD_EINVAL, "bad operand form");
  if (m < 0 || n < 0 || k < 0 || batch < 0) return fail(c, TSVD_EINVAL, "negative size");
  if (m == 0 || n == 0 || batch == 0) return TSVD_OK;
  if (!A || !B || !C) return fail(c, TSVD_EINVAL, "A, B and C must not be NULL");
  const int64_t ra = transa == TSVD_OP_N ? m : k, rb = transb == TSVD_OP_N ? k : n;
  if (lda < std::max<int64_t>(1, ra) || ldb < std::max<int64_t>(1, rb) ||
      ldc < std::max<int64_t>(1, m))
    return fail(c, TSVD_EINVAL, "leading dimension too small");
  if (batch > 1 && (stride_a < 0 || stride_b < 0 || stride_c < ldc * n))
    return fail(c, TSVD_EINVAL, "bad batch stride");
  if (batch > 65535) return fail(c, TSVD_EINVAL, "batch must be <= 65535");
  DeviceGuard dg(c->device);
  if (!dg.ok) return fail(c, TSVD_ECUDA, "cudaSetDevice(%d) failed", c->device);
  if (pointer_kind(A, c->device) != 0 || pointer_kind(B, c->device) != 0 ||
      pointer_kind(C, c->device) != 0)
    return fail(c, TSVD_EINVAL, "A, B and C must be device memory of the context's device");
  CGemm g;
  g.M = m;
  g.N = n;
  g.K = k;
  g.batch = batch;
  // op(A)(i, l)
  g.a.p = reinterpret_cast<const float2*>(A);
  g.a.idx = nullptr;
  g.a.bs = stride_a;
  g.a.s0 = transa == TSVD_OP_N ? 1 : lda;
  g.a.s1 = transa == TSVD_OP_N ? lda : 1;
  g.a.conj = transa == TSVD_OP_C;
  // op(B)(l, j)
  g.b.p = reinterpret_cast<const float2*>(B);
  g.b.idx = nullptr;
  g.b.bs = stride_b;
  g.b.s0 = transb == TSVD_OP_N ? 1 : ldb;
  g.b.s1 = transb == TSVD_OP_N ? ldb : 1;
  g.b.conj = transb == TSVD_OP_C;
  g.c.p = reinterpret_cast<const float2*>(C);
  g.c.idx = nullptr;
  g.c.bs = stride_c;
  g.c.s0 = 1;
  g.c.s1 = ldc;
  g.c.conj = 0;
  const int engine = c->opts.precision == TSVD_PRECISION_FP32 ? RSVT_GEMM_FP32 : rsvt_engine(c);
  TSVD_TRY(record_event(c, 0));
  TSVD_TRY(launch(c, launch_cgemm(g, engine, c->stream), "complex product"));
  TSVD_TRY(record_event(c, 0));
  return TSVD_OK;
}

}  // extern "C"
