// peak_probe.cu -- the measured FP32 CUDA-core throughput of a device: the denominator of the
// "alu" rooflines of the plain slice SVT (its Jacobi rotations and inner products run on the
// FP32 pipe, not the tensor cores).  A loop of independent fused multiply-adds per thread,
// scalar (fmaf) or packed FP32x2 (__ffma2_rn, the form the Jacobi kernels issue), timed with
// CUDA events on a private stream; the best of several launches is returned.
#include "tsvd.h"
#include "tsvd_internal.h"

#include <algorithm>

namespace {

constexpr int kChains = 8;      // independent accumulators per thread (hide the FMA latency)
constexpr int kIters = 2048;
constexpr int kThreads = 1024;

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(float* out, float a, float b) {
  if (PACKED) {
    float2 acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i)
      acc[i] = make_float2(1e-7f * threadIdx.x + (float)i, 1e-7f * blockIdx.x - (float)i);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i].x + acc[i].y;
    if (s == 1234.5f) out[0] = s;   // data-dependent store: the loop cannot be removed
  } else {
    float acc[2 * kChains];
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) acc[i] = 1e-7f * threadIdx.x + (float)i;
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
      for (int i = 0; i < 2 * kChains; ++i) acc[i] = fmaf(acc[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) s += acc[i];
    if (s == 1234.5f) out[0] = s;
  }
}

// Best TFLOP/s of `reps` timed launches (2 flops per FMA).
template <bool PACKED>
cudaError_t time_loop(cudaStream_t st, float* out, int blocks, int reps, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  const double flops = 2.0 * 2.0 * kChains * (double)kIters * kThreads * blocks;
  double best = 0.0;
  fma_loop_kernel<PACKED><<<blocks, kThreads, 0, st>>>(out, 0.9999999f, 1e-7f);   // warm-up
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    fma_loop_kernel<PACKED><<<blocks, kThreads, 0, st>>>(out, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" tsvd_status tsvd_measure_fp32_peak(int device, double* tflops_fma,
                                              double* tflops_fma2) {
  if (!tflops_fma || !tflops_fma2) return TSVD_EINVAL;
  *tflops_fma = *tflops_fma2 = 0.0;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ECUDA;
  }
  tsvd_status st = TSVD_OK;
  cudaStream_t s = nullptr;
  float* out = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&out, sizeof(float)) != cudaSuccess) {
    st = TSVD_ECUDA;
  } else {
    // two resident 1024-thread blocks per SM, eight waves' worth of blocks
    const int blocks = 16 * tsvd::device_sm_count();
    if (time_loop<false>(s, out, blocks, 5, tflops_fma) != cudaSuccess ||
        time_loop<true>(s, out, blocks, 5, tflops_fma2) != cudaSuccess)
      st = TSVD_ECUDA;
  }
  cudaGetLastError();
  if (out) cudaFree(out);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return st;
}
