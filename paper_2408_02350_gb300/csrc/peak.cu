// FP32 and FP64 fused-multiply-add throughput of the device, for the rooflines of
// the ALU-bound transport and of the plain FP64 path (measurement support, not part
// of the method): every thread runs 8 independent FMA chains (FP32 scalar or packed in
// pairs, or FP64), long enough that launch overhead is negligible; the host times the
// launch with events.
#include <cuda_runtime.h>

#include <cstdint>

#include "bgk.h"

namespace {

constexpr int CHAINS = 8;

template <bool PACKED>
__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float mul, float add) {
  const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 7);
  float acc = 0.0f;
  if (PACKED) {
    float2 a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = make_float2(seed + k, seed - k);
    const float2 m2 = make_float2(mul, mul), c2 = make_float2(add, add);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc += a[k].x + a[k].y;
  } else {
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = seed + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = fmaf(a[k], mul, add);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc += a[k];
  }
  if (acc == 12345.678f) out[0] = acc;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(256) k_dfma_peak(double* out, int iters, double mul, double add) {
  const double seed = 1.0 + 1e-3 * (double)(threadIdx.x & 7);
  double a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = seed + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], mul, add);
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) acc += a[k];
  if (acc == 12345.678) out[0] = acc;
}

}  // namespace

extern "C" int bgk_peak_fp64(double* dfma_per_s, void* stream) {
  if (!dfma_per_s) return BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BGK_E_CUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return BGK_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = 1 << 9;
  int st = BGK_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    k_dfma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = BGK_E_CUDA; break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (st == BGK_OK) *dfma_per_s = (double)blocks * threads * iters * CHAINS / (best * 1e-3);
  if (cudaGetLastError() != cudaSuccess) st = BGK_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}

extern "C" int bgk_peak_fp32(double* fma_per_s, double* fma2_per_s, int32_t* n_sm, void* stream) {
  if (!fma_per_s || !fma2_per_s || !n_sm) return BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BGK_E_CUDA;
  *n_sm = nsm;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return BGK_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = 1 << 14;
  int st = BGK_OK;
  for (int packed = 0; packed < 2 && st == BGK_OK; ++packed) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, s);
      if (packed) k_fma_peak<true><<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
      else k_fma_peak<false><<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = BGK_E_CUDA; break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    const double fmas = (double)blocks * threads * iters * CHAINS * (packed ? 2.0 : 1.0);
    (packed ? *fma2_per_s : *fma_per_s) = fmas / (best * 1e-3);
  }
  if (cudaGetLastError() != cudaSuccess) st = BGK_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
