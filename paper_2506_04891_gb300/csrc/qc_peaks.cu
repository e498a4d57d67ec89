// Arithmetic ceilings of the device, measured: scalar FP32 FMA, packed
// FP32x2 FMA (FFMA2) and FP64 FMA throughput.  The complex64 tile passes are
// built from FFMA2 / FFMA, the complex128 ones from DFMA, so these are the
// compute rooflines beside the measured HBM bandwidth (a complex128 layer pass
// needs about 16 FP64 flops per amplitude and gate, which the GPU's FP64 rate
// cannot feed at HBM speed).
//
// Each thread runs kChains independent FMA chains (enough to cover the
// pipeline latency) for `iters` iterations; the grid fills every SM.  The
// result of every chain is folded into one value that is written to a device
// sink only when it is impossible, so the work cannot be removed.
#include <cuda_runtime.h>

#include "../../include/qlayer.h"
#include "qc_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
__device__ double g_peak_sink;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float a, float b) {
  if constexpr (KIND == 0) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.2345e-30f) g_peak_sink = s;
  } else if constexpr (KIND == 1) {
    float2 v[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = make_float2((float)threadIdx.x, (float)c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
    if (s == -1.2345e-30f) g_peak_sink = s;
  } else {
    double v[kChains];
    const double ad = a, bd = b;
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], ad, bd);
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.2345e-30) g_peak_sink = s;
  }
}

}  // namespace

// kind 0: FP32 FFMA, 1: FP32x2 FFMA2 (two lanes per instruction), 2: FP64
// DFMA.  Writes the measured TFLOP/s (2 flops per FMA lane) to *tflops.
// Diagnostics: synchronises the device (it runs on a private stream and
// waits for it), allocates nothing.
extern "C" QC_API qc_status qc_fma_peak(int kind, double* tflops) {
  if (kind < 0 || kind > 2 || !tflops) return qc::set_error(QC_ERR_INVALID, "qc_fma_peak: kind 0..2, tflops non-NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return qc::set_error(QC_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return qc::set_error(QC_ERR_CUDA, cudaGetErrorString(e));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 8;  // 8 x 256 threads per SM: full occupancy at this register count
  const int iters = kind == 2 ? 1 << 12 : 1 << 16;
  auto launch = [&](int it) {
    if (kind == 0) k_peak<0><<<grid, kPeakThreads, 0, st>>>(it, 0.999f, 1e-7f);
    else if (kind == 1) k_peak<1><<<grid, kPeakThreads, 0, st>>>(it, 0.999f, 1e-7f);
    else k_peak<2><<<grid, kPeakThreads, 0, st>>>(it, 0.999f, 1e-7f);
  };
  launch(iters / 16);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return qc::set_error(QC_ERR_CUDA, cudaGetErrorString(e));
  const double lanes = kind == 1 ? 2.0 : 1.0;
  const double flops = 2.0 * lanes * (double)grid * kPeakThreads * kChains * (double)iters;
  *tflops = flops / (best * 1e-3) / 1e12;
  return QC_OK;
}
