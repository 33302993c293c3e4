// Device helpers: storage conversion, vector loads, block reductions, exact FP64 arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bgk_internal.cuh"

namespace bgk {

template <typename C> struct Pi;
template <> struct Pi<float> { static __device__ __forceinline__ float v() { return 3.14159265358979323846f; } };
template <> struct Pi<double> { static __device__ __forceinline__ double v() { return 3.14159265358979323846; } };

__device__ __forceinline__ float to_c(float v, float) { return v; }
__device__ __forceinline__ double to_c(double v, double) { return v; }

// ---- 4-wide loads and stores of the distribution (storage S, compute C) ----

__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  double2 a = reinterpret_cast<const double2*>(p)[0];
  double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float v[4]) {
  uint2 a = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&a.x);
  __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&a.y);
  float2 l = __bfloat1622float2(lo), h = __bfloat1622float2(hi);
  v[0] = l.x; v[1] = l.y; v[2] = h.x; v[3] = h.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float v[4]) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 a;
  a.x = *reinterpret_cast<uint32_t*>(&lo);
  a.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p) = a;
}

// scalar conversions
__device__ __forceinline__ double ld1(const double* p) { return *p; }
__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st1(double* p, double v) { *p = v; }
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// ---- FP64 arithmetic without fused multiply-add (matches a plain C evaluation) ----

__device__ __forceinline__ double sep_d(double xi, double xj, int periodic) {
  double d = __dadd_rn(xj, -xi);
  if (periodic) {
    if (d > 0.5) d = __dadd_rn(d, -1.0);
    else if (d < -0.5) d = __dadd_rn(d, 1.0);
  }
  return d;
}

template <int DIM>
__device__ __forceinline__ double dist2_d(const double* xi, const double* xj, int periodic) {
  double d2 = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double d = sep_d(xi[a], xj[a], periodic);
    d2 = __dadd_rn(d2, __dmul_rn(d, d));
  }
  return d2;
}

// ---- reductions ----

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a + b = s + e exactly (Knuth's two-sum; additions only, so nothing is contracted)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Sum of two unevaluated pairs (hi + lo): the high parts added exactly, the low parts and
// that addition's error added in FP32.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float bhi, float blo) {
  float s, e;
  two_sum(hi, bhi, s, e);
  hi = s;
  lo = (lo + blo) + e;
}

// Warp totals of N per-lane compensated FP32 sums (running sum s, compensation c: the
// lane's value is the unevaluated pair s + (-c)), combined in FP64.  Every lane gets the
// totals.  For N = 4 the sums are reduced transposed (FP64 runs at a small fraction of the
// FP32 rate, so the additions that involve all 32 lanes are kept few): at the step across
// 16 lanes a lane keeps two of the four sums and passes the other two, across 8 lanes
// one of its two, both as FP32 pairs with exact high-part additions; the pair is then
// converted to FP64 (exactly), the three last steps add in FP64, and lane 8 q, which holds
// the total of sum q, broadcasts it.  Otherwise each lane's pair is converted and the sums
// are reduced in FP64 one by one.
template <int N>
__device__ __forceinline__ void warp_total_f64(const float (&s)[N], const float (&c)[N], double (&out)[N]) {
  if constexpr (N == 4) {
    const int lane = threadIdx.x & 31;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    // keep sums (0, 1) below lane 16, (2, 3) from lane 16 on
    float k0h = hi16 ? s[2] : s[0], k0l = -(hi16 ? c[2] : c[0]);
    float k1h = hi16 ? s[3] : s[1], k1l = -(hi16 ? c[3] : c[1]);
    const float p0h = hi16 ? s[0] : s[2], p0l = -(hi16 ? c[0] : c[2]);
    const float p1h = hi16 ? s[1] : s[3], p1l = -(hi16 ? c[1] : c[3]);
    pair_add(k0h, k0l, __shfl_xor_sync(0xffffffffu, p0h, 16), __shfl_xor_sync(0xffffffffu, p0l, 16));
    pair_add(k1h, k1l, __shfl_xor_sync(0xffffffffu, p1h, 16), __shfl_xor_sync(0xffffffffu, p1l, 16));
    // keep the first of the two below lane 8 (mod 16), the second from lane 8 on
    float kh = hi8 ? k1h : k0h, kl = hi8 ? k1l : k0l;
    const float qh = hi8 ? k0h : k1h, ql = hi8 ? k0l : k1l;
    pair_add(kh, kl, __shfl_xor_sync(0xffffffffu, qh, 8), __shfl_xor_sync(0xffffffffu, ql, 8));
    double k = (double)kh + (double)kl;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = __shfl_sync(0xffffffffu, k, 8 * q);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = warp_sum((double)s[q] - (double)c[q]);
  }
}

// Sum NVAL per-thread values over the block.  Each warp reduces in T, the
// per-warp totals are combined in double.  Result valid in every thread.
// scratch: at least 32 * NVAL doubles of shared memory.
template <int NVAL, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NVAL], double (&out)[NVAL], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NVAL; ++q) {
    T s = warp_sum(v[q]);
    if (lane == 0) scratch[q * 32 + warp] = (double)s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NVAL; ++q) {
      double s = lane < nwarps ? scratch[q * 32 + lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) scratch[q * 32] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NVAL; ++q) out[q] = scratch[q * 32];
  __syncthreads();
}

__device__ __forceinline__ void set_status(DevStatus* st, int32_t bit) { atomicOr(&st->flags, bit); }

// Bounds-checked debug build (BGK_DEBUG_BOUNDS=1): an index j loaded from a list must lie
// in [0, n); a bad one is recorded (ST_BOUNDS) and replaced by `fallback`, an index that
// makes the access harmless (the point's own row, whose upwind term cancels).  The
// regular build returns j unchecked.
#ifndef BGK_DEBUG_BOUNDS
#define BGK_DEBUG_BOUNDS 0
#endif
__device__ __forceinline__ int checked_index(int j, int n, int fallback, DevStatus* st) {
#if BGK_DEBUG_BOUNDS
  if ((unsigned)j >= (unsigned)n) {
    set_status(st, ST_BOUNDS);
    return fallback;
  }
#endif
  (void)n; (void)fallback; (void)st;
  return j;
}
// The same for a list length m, which must lie in [0, cap] (a bad one becomes 0).
__device__ __forceinline__ int checked_count(int m, int cap, DevStatus* st) {
#if BGK_DEBUG_BOUNDS
  if (m < 0 || m > cap) {
    set_status(st, ST_BOUNDS);
    return 0;
  }
#endif
  (void)cap; (void)st;
  return m;
}

}  // namespace bgk
