// Per-step kernels of the meshfree BGK scheme (Sec. 3.2, 3.4.2, 5).
//
// k_transport: one CTA per interior point i; each thread owns NCH chunks of 4
//   consecutive velocities.  The neighbour list and stencil of i are staged
//   in shared memory; for every neighbour j the thread reads f_j for its
//   velocities (16-byte loads, a warp reads 512 contiguous bytes per chunk)
//   and accumulates
//     m_ij(v) = sum_d min(c.P_d, 0),  acc += m_ij f_j,  sk += m_ij,
//   with c = v - U_i^n (ALE) or v.  Since the upwind coefficient is
//   K_ij = sum_d (c.P_d - |c.P_d|) = 2 m_ij, the transported value is
//     f~_i = f_i - dt sum_j K_ij (f_j - f_i) = f_i - 2 dt (acc - sk f_i).
//   The same CTA then sums the moments of f~_i over all velocities (warp
//   shuffles, cross-warp totals in double by one thread), forms rho, U, T,
//   tau and the Maxwellian, and writes f^{n+1} = (tau f~ + dt M)/(tau + dt)
//   to the other buffer: one read of f_i, neighbour reads served mostly from
//   L2, one write of f_i^{n+1}.
// k_walls: one CTA per wall point; arriving velocities (v.n <= 0) get the WLS
//   reconstruction from interior f^{n+1}; leaving velocities get
//   rho_w M_w(v) with rho_w from zero net mass flux.
// k_move: x += dt U^{n+1} at interior points (FP64, no fused multiply-add).
#include <algorithm>
#include <type_traits>

#include "bgk_internal.cuh"
#include "device_common.cuh"
#include "motion.cuh"
#include "transport_wp.cuh"
#include "transport_stage.cuh"

namespace bgk {

static inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// Fixed points: pair each velocity with its mirror in the transport (1) or not (0).
#ifndef BGK_TRANSPORT_MIRROR
#define BGK_TRANSPORT_MIRROR 1
#endif
__host__ __device__ static inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

constexpr int RED_BYTES = 32 * 8 * 8;   // block-reduction scratch: 8 values x 32 warps, double
constexpr int NODE_BYTES = 64 * 8;      // velocity nodes, up to 64 per axis

// Finalise the moments from raw sums R = sum g, Mx = sum v g, E = sum |v|^2 g (+ sum h)
// (quadrature weight dv^dim applied to rho only; it cancels in U and T).
template <int DIM>
__device__ __forceinline__ void finish_moments(const double* tot, double wv, double* rho, double* U, double* T) {
  const double R = tot[0];
  double u2 = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) { U[a] = tot[1 + a] / R; u2 += U[a] * U[a]; }
  *T = (tot[DIM + 1] - R * u2) / (3.0 * R);
  *rho = R * wv;
}

template <typename C>
__device__ __forceinline__ C expc(C x);
template <> __device__ __forceinline__ float expc<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double expc<double>(double x) { return exp(x); }

template <typename C> __device__ __forceinline__ C minc(C a, C b);
template <> __device__ __forceinline__ float minc<float>(float a, float b) { return fminf(a, b); }
template <> __device__ __forceinline__ double minc<double>(double a, double b) { return fmin(a, b); }

// Sum NVAL per-thread values: warp shuffles in T, then thread 0 adds the warp
// totals in double.  Result in out[] of every thread.
template <int NVAL, typename T>
__device__ __forceinline__ void block_sum0(const T (&v)[NVAL], double (&out)[NVAL], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NVAL; ++q) {
    T s = warp_sum(v[q]);
    if (lane == 0) scratch[q * 32 + warp] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NVAL; ++q) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += scratch[q * 32 + w];
      scratch[q * 32] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NVAL; ++q) out[q] = scratch[q * 32];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// transport + moments + relaxation
// ---------------------------------------------------------------------------
// Moments of f~_i from the raw sums tot, tau and the Maxwellian (one thread, FP64,
// broadcast through shared memory), then f^{n+1} = (tau f~ + dt M)/(tau + dt) (RK = 1:
// the exact relaxation over dt/2) for the thread's chunks, written to the output row.
// vk0: first grid velocity of the row.
template <typename S, typename C, int DIM, int NCH, int RK = 0>
__device__ __forceinline__ void relax_cta(const CaseView& cv, const int i, const double (&tot)[DIM + 2],
                                          const C (&ft)[NCH][DIM == 2 ? 2 : 1][4], const C* s_v, double* s_red,
                                          const int vk0) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int nchunk = NVp >> 2;
  const int64_t rowlen = (int64_t)NC * NVp;
  // moments, tau and relaxation coefficients (one thread, FP64), broadcast through shared memory
  C* s_fin = reinterpret_cast<C*>(s_red + 6 * 32);  // past the slots block_sum0 uses (5 x 32)
  if (threadIdx.x == 0) {
    double rho, Un[3] = {0, 0, 0}, T;
    const double wv = cv.wv;
    finish_moments<DIM>(tot, wv, &rho, Un, &T);
    double* mo = cv.mom + (int64_t)i * MOM_STRIDE;
    mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
    double a = 1.0, b = 0.0, pref = 0.0, inv2T = 0.0;
    if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T)) {
      set_status(cv.status, ST_NONFINITE);
    } else if (cv.tau_mode != 2) {
      const double pi = 3.14159265358979323846;
      const double tau = cv.tau_mode == 1 ? sqrt(2.0 / pi) * cv.kn : sqrt(2.0 / pi) * cv.kn / (rho * sqrt(T));
      if (RK == 1) {
        a = exp(-0.5 * cv.dt / tau);
        b = -expm1(-0.5 * cv.dt / tau);
      } else {
        a = tau / (tau + cv.dt);
        b = cv.dt / (tau + cv.dt);
      }
      pref = DIM == 2 ? rho / (2.0 * pi * T) : rho / pow(2.0 * pi * T, 1.5);
      inv2T = 1.0 / (2.0 * T);
    }
    s_fin[0] = (C)a; s_fin[1] = (C)b; s_fin[2] = (C)pref; s_fin[3] = (C)inv2T; s_fin[4] = (C)T;
#pragma unroll
    for (int d = 0; d < DIM; ++d) s_fin[5 + d] = (C)Un[d];
  }
  __syncthreads();
  const C ca = s_fin[0], cb = s_fin[1], pref = s_fin[2], inv2T = s_fin[3], Tn = s_fin[4];
  C Un[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) Un[d] = s_fin[5 + d];

  S* fo = reinterpret_cast<S*>(cv.f_out) + (int64_t)i * rowlen;
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int chunk = threadIdx.x + q * blockDim.x;
    if (chunk < nchunk) {
      C out[NC][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 4 * chunk + e;
        if (k < NV) {
          int kk = k + vk0;
          C c2 = (C)0;
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const C d = s_v[kk % nv] - Un[a];
            kk /= nv;
            c2 += d * d;
          }
          const C M = pref * expc<C>(-c2 * inv2T);
          out[0][e] = ca * ft[q][0][e] + cb * M;
          if (NC == 2) out[NC - 1][e] = ca * ft[q][NC - 1][e] + cb * Tn * M;
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) out[c][e] = (C)0;
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) st4(fo + (int64_t)c * NVp + 4 * chunk, out[c]);
    }
  }
}

template <typename S, typename C, int DIM, int NCH, bool ALE, bool SH = false, bool AVG = false>
__global__ void __launch_bounds__(256) k_transport(const CaseView cv) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_red = reinterpret_cast<double*>(smem);
  C* s_v = reinterpret_cast<C*>(smem + RED_BYTES);
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + RED_BYTES + NODE_BYTES);
  C* s_P = reinterpret_cast<C*>(smem + RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * cv.cap));

  const int i = cv.int_idx[blockIdx.x];
  const int m = checked_count(cv.cnt[i], cv.cap, cv.status);
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int nchunk = NVp >> 2;
  const int vk0 = SH ? cv.vk0 : 0;
  {
    const int32_t* col = cv.col + (int64_t)i * cv.cap;
    const C* P = reinterpret_cast<const C*>(cv.P) + (int64_t)i * cv.cap * DD;
    for (int t = threadIdx.x; t < m; t += blockDim.x) s_col[t] = checked_index(col[t], cv.n, i, cv.status);
    for (int t = threadIdx.x; t < m * DD; t += blockDim.x) s_P[t] = P[t];
    for (int t = threadIdx.x; t < nv; t += blockDim.x) s_v[t] = (C)cv.vnodes[t];
  }
  __syncthreads();

  C U[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) U[a] = ALE ? (C)cv.mom[(int64_t)i * MOM_STRIDE + 1 + a] : (C)0;

  // convective velocities c = v - U of this thread's velocities
  C cvel[NCH][4][DIM];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int chunk = threadIdx.x + q * blockDim.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * chunk + e;
      int kk = k < NV ? k + vk0 : 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        cvel[q][e][a] = k < NV ? s_v[kk % nv] - U[a] : (C)0;
        kk /= nv;
      }
    }
  }

  C acc[NCH][NC][4], sk[NCH][4];
#pragma unroll
  for (int q = 0; q < NCH; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      sk[q][e] = (C)0;
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[q][c][e] = (C)0;
    }

  const S* fbase = reinterpret_cast<const S*>(cv.f_in);
  const int64_t rowlen = (int64_t)NC * NVp;
  for (int s = 0; s < m; ++s) {
    const int j = s_col[s];
    C P[DD];
#pragma unroll
    for (int t = 0; t < DD; ++t) P[t] = s_P[s * DD + t];
    const S* fj = fbase + (int64_t)j * rowlen;
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int chunk = threadIdx.x + q * blockDim.x;
      if (chunk < nchunk) {
        C fv[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c) ld4(fj + (int64_t)c * NVp + 4 * chunk, fv[c]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          C mk = (C)0;
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            C p = cvel[q][e][0] * P[d * DIM + 0];
#pragma unroll
            for (int a = 1; a < DIM; ++a) p += cvel[q][e][a] * P[d * DIM + a];
            mk += minc(p, (C)0);
          }
          sk[q][e] += mk;
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[q][c][e] += mk * fv[c][e];
        }
      }
    }
  }

  // f~ = f_i - 2 dt (acc - sk f_i) and one-pass raw moment sums
  const S* fi = fbase + (int64_t)i * rowlen;
  const C two_dt = (C)(2.0 * cv.dt);
  C ft[NCH][NC][4];
  C part[DIM + 2];
#pragma unroll
  for (int t = 0; t < DIM + 2; ++t) part[t] = (C)0;
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int chunk = threadIdx.x + q * blockDim.x;
    if (chunk < nchunk) {
      C fiv[NC][4], fav[NC][4];
#pragma unroll
      for (int c = 0; c < NC; ++c) ld4(fi + (int64_t)c * NVp + 4 * chunk, fiv[c]);
      if (AVG) {
        const S* fa = reinterpret_cast<const S*>(cv.f_avg) + (int64_t)i * rowlen;
#pragma unroll
        for (int c = 0; c < NC; ++c) ld4(fa + (int64_t)c * NVp + 4 * chunk, fav[c]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int c = 0; c < NC; ++c) ft[q][c][e] = fiv[c][e] - two_dt * (acc[q][c][e] - sk[q][e] * fiv[c][e]);
        if (AVG) {
#pragma unroll
          for (int c = 0; c < NC; ++c) ft[q][c][e] = (C)0.5 * (ft[q][c][e] + fav[c][e]);
        }
        const int k = 4 * chunk + e;
        if (k < NV) {
          int kk = k + vk0;
          C v2 = (C)0;
          const C g = ft[q][0][e];
          part[0] += g;
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const C va = s_v[kk % nv];
            kk /= nv;
            part[1 + a] += va * g;
            v2 += va * va;
          }
          part[DIM + 1] += v2 * g;
          if (NC == 2) part[DIM + 1] += ft[q][NC - 1][e];
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int c = 0; c < NC; ++c) ft[q][c][e] = (C)0;
    }
  }
  double tot[DIM + 2];
  block_sum0<DIM + 2, C>(part, tot, s_red);

  if constexpr (SH) {
    // sharded step: the slab's sums to the exchange buffer, f~ to the output row
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < DIM + 2; ++q) cv.xs[(int64_t)i * (DIM + 2) + q] = tot[q];
    }
    S* fo = reinterpret_cast<S*>(cv.f_out) + (int64_t)i * rowlen;
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int chunk = threadIdx.x + q * blockDim.x;
      if (chunk < nchunk) {
#pragma unroll
        for (int c = 0; c < NC; ++c) st4(fo + (int64_t)c * NVp + 4 * chunk, ft[q][c]);
      }
    }
  } else {
    relax_cta<S, C, DIM, NCH, AVG ? 1 : 0>(cv, i, tot, ft, s_v, s_red, 0);
  }
}

template <typename S, typename C, int DIM, int NCH, bool SH = false, bool AVG = false>
static void launch_transport_t(const CaseView& cv, int threads, size_t smem, cudaStream_t s) {
  if (AVG) {
    // the second-order step is for fixed points
    auto k = k_transport<S, C, DIM, NCH, false, false, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<cv.n_int, threads, smem, s>>>(cv);
  } else if (cv.ale) {
    auto k = k_transport<S, C, DIM, NCH, true, SH>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<cv.n_int, threads, smem, s>>>(cv);
  } else {
    auto k = k_transport<S, C, DIM, NCH, false, SH>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<cv.n_int, threads, smem, s>>>(cv);
  }
}

// Sharded step, FP64 storage: one CTA per interior point (the launch shape of
// k_transport) relaxes f~ in the output row with the moments of the summed sums.
template <typename S, typename C, int DIM, int NCH>
__global__ void __launch_bounds__(256) k_shard_relax_cta(const CaseView cv) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  __shared__ double s_red[8 * 32];
  __shared__ C s_v[64];
  const int i = cv.int_idx[blockIdx.x];
  const int NVp = cv.NVp, nchunk = NVp >> 2;
  for (int t = threadIdx.x; t < cv.nv; t += blockDim.x) s_v[t] = (C)cv.vnodes[t];
  const S* fo = reinterpret_cast<const S*>(cv.f_out) + (int64_t)i * NC * NVp;
  C ft[NCH][NC][4];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int chunk = threadIdx.x + q * blockDim.x;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (chunk < nchunk) {
        ld4(fo + (int64_t)c * NVp + 4 * chunk, ft[q][c]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) ft[q][c][e] = (C)0;
      }
    }
  }
  double tot[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) tot[q] = cv.xs[(int64_t)i * (DIM + 2) + q];
  __syncthreads();
  relax_cta<S, C, DIM, NCH>(cv, i, tot, ft, s_v, s_red, cv.vk0);
}

// CTA shape of the FP64 transport: NCH chunks of 4 velocities per thread, at most 256 threads.
static inline void cta_shape(int NVp, int* nch, int* threads) {
  const int nchunk = NVp / 4;
  int q = 1;
  while ((nchunk + q - 1) / q > 256) q *= 2;
  *nch = q;
  *threads = (((nchunk + q - 1) / q) + 31) / 32 * 32;
}

template <typename S, typename C, int DIM, bool SH = false, bool AVG = false>
static void launch_transport_d(const CaseView& cv, cudaStream_t s) {
  int nch, threads;
  cta_shape(cv.NVp, &nch, &threads);
  const size_t smem = RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * cv.cap) + sizeof(C) * cv.cap * DIM * DIM;
  switch (nch) {
    case 1: launch_transport_t<S, C, DIM, 1, SH, AVG>(cv, threads, smem, s); break;
    case 2: launch_transport_t<S, C, DIM, 2, SH, AVG>(cv, threads, smem, s); break;
    case 4: launch_transport_t<S, C, DIM, 4, SH, AVG>(cv, threads, smem, s); break;
    default: launch_transport_t<S, C, DIM, 8, SH, AVG>(cv, threads, smem, s); break;
  }
}

// Second-order step, FP64 storage: the exact relaxation over dt/2 of the output row of
// each interior point in place, with the moments of that row (one CTA per point).
template <typename S, typename C, int DIM, int NCH>
__global__ void __launch_bounds__(256) k_relax_half_cta(const CaseView cv) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  __shared__ double s_red[8 * 32];
  __shared__ C s_v[64];
  const int i = cv.int_idx[blockIdx.x];
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp, nchunk = NVp >> 2;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_v[t] = (C)cv.vnodes[t];
  __syncthreads();
  const S* fo = reinterpret_cast<const S*>(cv.f_out) + (int64_t)i * NC * NVp;
  C ft[NCH][NC][4];
  C part[DIM + 2];
#pragma unroll
  for (int t = 0; t < DIM + 2; ++t) part[t] = (C)0;
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int chunk = threadIdx.x + q * blockDim.x;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (chunk < nchunk) {
        ld4(fo + (int64_t)c * NVp + 4 * chunk, ft[q][c]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) ft[q][c][e] = (C)0;
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * chunk + e;
      if (chunk < nchunk && k < NV) {
        int kk = k;
        C v2 = (C)0;
        const C g = ft[q][0][e];
        part[0] += g;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const C va = s_v[kk % nv];
          kk /= nv;
          part[1 + a] += va * g;
          v2 += va * va;
        }
        part[DIM + 1] += v2 * g;
        if (NC == 2) part[DIM + 1] += ft[q][NC - 1][e];
      }
    }
  }
  double tot[DIM + 2];
  block_sum0<DIM + 2, C>(part, tot, s_red);
  relax_cta<S, C, DIM, NCH, 1>(cv, i, tot, ft, s_v, s_red, 0);
}

template <typename S, typename C, int DIM>
static void launch_shard_relax_d(const CaseView& cv, cudaStream_t s) {
  int nch, threads;
  cta_shape(cv.NVp, &nch, &threads);
  switch (nch) {
    case 1: k_shard_relax_cta<S, C, DIM, 1><<<cv.n_int, threads, 0, s>>>(cv); break;
    case 2: k_shard_relax_cta<S, C, DIM, 2><<<cv.n_int, threads, 0, s>>>(cv); break;
    case 4: k_shard_relax_cta<S, C, DIM, 4><<<cv.n_int, threads, 0, s>>>(cv); break;
    default: k_shard_relax_cta<S, C, DIM, 8><<<cv.n_int, threads, 0, s>>>(cv); break;
  }
}

// Shared memory of the warp-per-point kernels with W warps: velocity nodes, lists,
// stencils, compensated moment sums.
template <int DIM>
__host__ __device__ inline size_t wp_smem_bytes(int W, int cap) {
  return 256 * W + align16(sizeof(int32_t) * cap * W) + align16(sizeof(float) * cap * DIM * DIM * W) +
         sizeof(float) * kahan_floats<DIM>() * W;
}

// Warps per CTA of the single-case first-order launch.  The CTA's points are consecutive
// in Morton order, but a smaller CTA loses less to the uneven neighbour counts of its
// warps (201^2 x 32^2 ALE cavity, transport ms: 1 warp 0.441, 2 0.440, 4 0.436, 8 0.440,
// 16 0.453, 32 0.503).
#ifndef BGK_WP_WARPS
#define BGK_WP_WARPS 4
#endif
template <typename S, int DIM, bool ALE, bool ROW, int VPL, bool SH = false, bool AVG = false>
__global__ void __launch_bounds__(32 * BGK_WP_WARPS, VPL == 4 ? 32 / BGK_WP_WARPS : 16 / BGK_WP_WARPS)
    k_transport_wp(const CaseView cv) {
  constexpr int DD = DIM * DIM;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int cap = cv.cap;
  float* s_v = reinterpret_cast<float*>(smem) + warp * 64;
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + 256 * W) + warp * cap;
  float* s_P0 = reinterpret_cast<float*>(smem + 256 * W + align16(sizeof(int32_t) * cap * W));
  float* s_P = s_P0 + (size_t)warp * cap * DD;
  float* s_k = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s_P0) + align16(sizeof(float) * W * cap * DD)) +
               warp * kahan_floats<DIM>();
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  transport_point_wp<S, DIM, ALE, ROW, VPL, VPL == 4, SH, AVG>(cv, cv.int_idx[t], s_v, s_col, s_P, s_k);
}

// Staged variant (2D, FP32, nv % 4 == 0): the neighbour rows come through per-warp rings
// of bulk copies instead of L1 (transport_stage.cuh).
#ifndef BGK_WP_STAGE
#define BGK_WP_STAGE 0
#endif
#ifndef BGK_STAGE_MINB
#define BGK_STAGE_MINB (32 / BGK_WP_WARPS)
#endif
template <bool ALE>
__global__ void __launch_bounds__(32 * BGK_WP_WARPS, BGK_STAGE_MINB) k_transport_stage(const CaseView cv) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int cap = cv.cap;
  float* s_v = reinterpret_cast<float*>(smem) + warp * 64;
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + 256 * W) + warp * cap;
  float* s_P0 = reinterpret_cast<float*>(smem + 256 * W + align16(sizeof(int32_t) * cap * W));
  float* s_P = s_P0 + (size_t)warp * cap * 4;
  float* s_k = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s_P0) + align16(sizeof(float) * W * cap * 4)) +
               warp * kahan_floats<2>();
  unsigned char* ring0 = smem + stage_ring_offset(wp_smem_bytes<2>(W, cap));
  float* s_ring = reinterpret_cast<float*>(ring0 + (size_t)warp * kStageD * kStageG * kStageRowBytes);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(ring0 + (size_t)W * kStageD * kStageG * kStageRowBytes) + warp * kStageD;
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  transport_point_stage<ALE>(cv, cv.int_idx[t], s_v, s_col, s_P, s_k, s_ring, s_bar);
}

// Second-order step, FP32/BF16 storage: one warp per interior point relaxes its output
// row exactly over dt/2 in place, with the moments of that row (compensated lane sums).
template <typename S, int DIM, bool ROW>
__global__ void __launch_bounds__(256) k_relax_half_wp(const CaseView cv) {
  constexpr int NC = DIM == 2 ? 2 : 1, VPL = 4;
  __shared__ __align__(16) float s_vall[8 * 64];  // chunk_velocities reads groups of 4
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_v = s_vall + warp * 64;
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  for (int q = lane; q < cv.nv; q += 32) s_v[q] = cv.vnodes_f[q];
  __syncwarp();
  const int i = cv.int_idx[t];
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const float inv_nv = 1.0f / (float)nv;
  const S* fi = reinterpret_cast<const S*>(cv.f_out) + (int64_t)i * NC * NVp;
  float msum[DIM + 2], mcmp[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) { msum[q] = 0.0f; mcmp[q] = 0.0f; }
  for (int chunk = lane; chunk * VPL < NVp; chunk += 32) {
    const int k0 = chunk * VPL;
    float vel[VPL][DIM];
    bool kin[VPL];
    chunk_velocities<DIM, VPL, ROW>(k0, nv, NV, inv_nv, s_v, vel, kin);
    float g[NC][VPL];
#pragma unroll
    for (int c = 0; c < NC; ++c) ldv<S, VPL>(fi + (int64_t)c * NVp + k0, g[c]);
    float ps[DIM + 2];
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) ps[q] = 0.0f;
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
      const float g0 = kin[e] ? g[0][e] : 0.0f;
      float v2 = 0.0f;
      ps[0] += g0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { ps[1 + a] = fmaf(vel[e][a], g0, ps[1 + a]); v2 = fmaf(vel[e][a], vel[e][a], v2); }
      ps[DIM + 1] = fmaf(v2, g0, ps[DIM + 1]);
      if (NC == 2) ps[DIM + 1] += kin[e] ? g[NC - 1][e] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) {
      const float y = ps[q] - mcmp[q];
      const float tt = msum[q] + y;
      mcmp[q] = (tt - msum[q]) - y;
      msum[q] = tt;
    }
  }
  finish_point<S, DIM, ROW, VPL, 1>(cv, i, s_v, msum, mcmp);
}

// Sharded step, FP32/BF16 storage: one warp per interior point relaxes f~ in the
// output row with the moments of the summed sums (the relaxation of k_transport_wp).
template <typename S, int DIM, bool ROW>
__global__ void __launch_bounds__(256) k_shard_relax_wp(const CaseView cv) {
  __shared__ __align__(16) float s_vall[8 * 64];  // chunk_velocities reads groups of 4
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_v = s_vall + warp * 64;
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  for (int q = lane; q < cv.nv; q += 32) s_v[q] = cv.vnodes_f[q];
  __syncwarp();
  const int i = cv.int_idx[t];
  double tot[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) tot[q] = cv.xs[(int64_t)i * (DIM + 2) + q];
  relax_point<S, DIM, ROW, 4, true>(cv, i, s_v, tot);
}

// Fixed points with a mirror-symmetric velocity grid (nv % 4 == 0, NV % 8 == 0): one
// warp per interior point, each lane a velocity chunk and its mirror chunk; 79
// registers, 24 warps per SM.  Used in 3D, where it saves a quarter of the
// per-neighbour instructions (41^3 x 16^3 cavity: 6.63 against 7.50 ms per step with
// the 8-velocity kernel); in 2D the extra registers cost more than the saved
// instructions (201^2 x 32^2 fixed points: 0.483 ms at 4 CTAs per SM with spills,
// 0.561 ms at 3, against 0.447 ms), so 2D keeps the plain kernel.
#ifndef BGK_MIRROR_MIN_BLOCKS
#define BGK_MIRROR_MIN_BLOCKS 3
#endif
template <typename S, int DIM, bool KS>
__global__ void __launch_bounds__(256, BGK_MIRROR_MIN_BLOCKS) k_transport_mirror(const CaseView cv) {
  constexpr int DD = DIM * DIM;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int cap = cv.cap;
  float* s_v = reinterpret_cast<float*>(smem) + warp * 64;
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + 256 * W) + warp * cap;
  float* s_P0 = reinterpret_cast<float*>(smem + 256 * W + align16(sizeof(int32_t) * cap * W));
  float* s_P = s_P0 + (size_t)warp * cap * DD;
  float* s_k = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s_P0) + align16(sizeof(float) * W * cap * DD)) +
               warp * kahan_floats<DIM>();
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  transport_point_mirror<S, DIM, KS>(cv, cv.int_idx[t], s_v, s_col, s_P, s_k);
}

// Many cases in one persistent launch: items[k] = (case, interior slot), tiles of W
// consecutive items per CTA, tiles taken in grid-stride order.  Every warp reads
// its case's descriptor; the ROW4 variant is chosen per warp.
// 3 CTAs per SM (80 registers, 8 bytes spilled) beats 2 (114 registers, no spills) on
// the 64-cavity sweep: 4.54 against 4.99 ms per step (when measured); the compensated
// sums in shared memory (KS, as the single-case kernel) lose here: 4.46 ms at 3 CTAs per
// SM and 4.57 ms at 4 against 4.04 ms.
#ifndef BGK_BATCH_KS
#define BGK_BATCH_KS false
#endif
#ifndef BGK_BATCH_MIN_BLOCKS
#define BGK_BATCH_MIN_BLOCKS 3
#endif
template <typename S, int DIM>
__global__ void __launch_bounds__(256, BGK_BATCH_MIN_BLOCKS) k_transport_batch(const CaseView* __restrict__ cases, const int2* __restrict__ items,
                                                             int n_items, int capmax) {
  constexpr int DD = DIM * DIM;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
  float* s_v = reinterpret_cast<float*>(smem) + warp * 64;
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + 256 * W) + warp * capmax;
  float* s_P0 = reinterpret_cast<float*>(smem + 256 * W + align16(sizeof(int32_t) * capmax * W));
  float* s_P = s_P0 + (size_t)warp * capmax * DD;
  float* s_k = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s_P0) + align16(sizeof(float) * W * capmax * DD)) +
               warp * kahan_floats<DIM>();
  for (int tile = blockIdx.x; tile * W < n_items; tile += gridDim.x) {
    const int it = tile * W + warp;
    if (it >= n_items) continue;
    const int2 e = items[it];
    const CaseView& cv = cases[e.x];
    const int i = cv.int_idx[e.y];
    // (batched stepping takes fixed points only: c = v)
    if (cv.nv % 4 == 0) transport_point_wp<S, DIM, false, true, 4, BGK_BATCH_KS>(cv, i, s_v, s_col, s_P, s_k);
    else transport_point_wp<S, DIM, false, false, 4, BGK_BATCH_KS>(cv, i, s_v, s_col, s_P, s_k);
    __syncwarp();
  }
}

// Velocities per lane: 8 in 3D when the velocity rows split into groups of 8 (fewer
// per-neighbour instructions and more loads in flight pay off there: 7.1 vs 8.6 ms
// on the 41^3 x 16^3 cavity), 4 in 2D (where the lower occupancy of the wider
// variant costs more than it saves: 0.53 vs 0.48 ms on the 201^2 x 32^2 cavity).
int transport_vpl = 0;  // 0 = automatic; 4 or 8 forces a width

template <typename S, int DIM>
static void launch_transport_wp(const CaseView& cv, cudaStream_t s) {
  const int W = BGK_WP_WARPS, threads = 32 * W;
  const size_t smem = wp_smem_bytes<DIM>(W, cv.cap);
  const int grid = (cv.n_int + W - 1) / W;
  const bool row4 = cv.nv % 4 == 0, row8 = cv.nv % 8 == 0 && cv.NVp % 8 == 0;
  if constexpr (DIM == 3) {
    if (BGK_TRANSPORT_MIRROR && !cv.ale && row4 && cv.NV % 8 == 0) {
      auto k = k_transport_mirror<S, DIM, false>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k<<<grid, threads, smem, s>>>(cv);
      return;
    }
  }
  const bool v8 = transport_vpl == 8 ? (cv.NVp % 8 == 0) : (transport_vpl == 4 ? false : (DIM == 3 && row8));
  if constexpr (BGK_WP_STAGE && DIM == 2 && std::is_same<S, float>::value) {
    // (bulk copies need 16-byte aligned rows: caller-bound storage may start anywhere)
    if (row4 && !v8 && cv.NVp % 4 == 0 && (reinterpret_cast<uintptr_t>(cv.f_in) & 15) == 0) {
      const size_t ssm = stage_smem_bytes(smem, W);
      auto k = cv.ale ? k_transport_stage<true> : k_transport_stage<false>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
      k<<<grid, threads, ssm, s>>>(cv);
      return;
    }
  }
#define BGK_LAUNCH_WP(ALE, ROW, VPL)                                                      \
  {                                                                                       \
    auto k = k_transport_wp<S, DIM, ALE, ROW, VPL>;                                       \
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    k<<<grid, threads, smem, s>>>(cv);                                                    \
  }
  if (v8) {
    if (cv.ale) {
      if (row8) BGK_LAUNCH_WP(true, true, 8) else BGK_LAUNCH_WP(true, false, 8)
    } else {
      if (row8) BGK_LAUNCH_WP(false, true, 8) else BGK_LAUNCH_WP(false, false, 8)
    }
  } else if (cv.ale) {
    if (row4) BGK_LAUNCH_WP(true, true, 4) else BGK_LAUNCH_WP(true, false, 4)
  } else {
    if (row4) BGK_LAUNCH_WP(false, true, 4) else BGK_LAUNCH_WP(false, false, 4)
  }
#undef BGK_LAUNCH_WP
}

int launch_transport_fp32(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 1) launch_transport_wp<float, 2>(cv, s);
    else launch_transport_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 1) launch_transport_wp<float, 3>(cv, s);
    else launch_transport_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

template <typename S, int DIM>
static void launch_transport_avg_wp(const CaseView& cv, cudaStream_t s) {
  const int W = BGK_WP_WARPS, threads = 32 * W;
  const size_t smem = wp_smem_bytes<DIM>(W, cv.cap);
  const int grid = (cv.n_int + W - 1) / W;
  if (cv.nv % 4 == 0) {
    auto k = k_transport_wp<S, DIM, false, true, 4, false, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, threads, smem, s>>>(cv);
  } else {
    auto k = k_transport_wp<S, DIM, false, false, 4, false, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, threads, smem, s>>>(cv);
  }
}

int launch_transport_avg(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) launch_transport_d<double, double, 2, false, true>(cv, s);
    else if (cv.storage == 1) launch_transport_avg_wp<float, 2>(cv, s);
    else launch_transport_avg_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 0) launch_transport_d<double, double, 3, false, true>(cv, s);
    else if (cv.storage == 1) launch_transport_avg_wp<float, 3>(cv, s);
    else launch_transport_avg_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

template <typename S, typename C, int DIM>
static void launch_relax_half_d(const CaseView& cv, cudaStream_t s) {
  int nch, threads;
  cta_shape(cv.NVp, &nch, &threads);
  switch (nch) {
    case 1: k_relax_half_cta<S, C, DIM, 1><<<cv.n_int, threads, 0, s>>>(cv); break;
    case 2: k_relax_half_cta<S, C, DIM, 2><<<cv.n_int, threads, 0, s>>>(cv); break;
    case 4: k_relax_half_cta<S, C, DIM, 4><<<cv.n_int, threads, 0, s>>>(cv); break;
    default: k_relax_half_cta<S, C, DIM, 8><<<cv.n_int, threads, 0, s>>>(cv); break;
  }
}

template <typename S, int DIM>
static void launch_relax_half_wp(const CaseView& cv, cudaStream_t s) {
  const int W = 8, grid = (cv.n_int + W - 1) / W;
  if (cv.nv % 4 == 0) k_relax_half_wp<S, DIM, true><<<grid, 32 * W, 0, s>>>(cv);
  else k_relax_half_wp<S, DIM, false><<<grid, 32 * W, 0, s>>>(cv);
}

int launch_relax_half(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0 || cv.tau_mode == 2) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) launch_relax_half_d<double, double, 2>(cv, s);
    else if (cv.storage == 1) launch_relax_half_wp<float, 2>(cv, s);
    else launch_relax_half_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 0) launch_relax_half_d<double, double, 3>(cv, s);
    else if (cv.storage == 1) launch_relax_half_wp<float, 3>(cv, s);
    else launch_relax_half_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

int launch_transport(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) launch_transport_d<double, double, 2>(cv, s);
    else if (cv.storage == 1) launch_transport_wp<float, 2>(cv, s);
    else launch_transport_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 0) launch_transport_d<double, double, 3>(cv, s);
    else if (cv.storage == 1) launch_transport_wp<float, 3>(cv, s);
    else launch_transport_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

// ---------------------------------------------------------------------------
// walls
// ---------------------------------------------------------------------------
// The per-wall-point body (one CTA), shared by the single-case and batched kernels.
// PH = 0: the whole step.  The sharded step splits it around the sum over all slabs:
// PH = 1 writes the arriving half and the wall sums of the slab to cv.xs[w][2 dim + 6]
//   [0] sum_{arriving} |c_n| g   [1] sum_{leaving} c_n M_w   [2, dim + 4) moment sums of
//   the arriving half   [dim + 4, 2 dim + 6) moment sums of M_w over the leaving half;
// PH = 2 reads the summed cv.xs, writes rho_w M_w to the leaving half and the moments.
template <int DIM>
__host__ __device__ constexpr int wall_sums() { return 2 * DIM + 6; }

template <typename S, typename C, int DIM, int PH = 0>
__device__ __forceinline__ void walls_point(const CaseView& cv, const int w, unsigned char* smem) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  double* s_red = reinterpret_cast<double*>(smem);
  C* s_v = reinterpret_cast<C*>(smem + RED_BYTES);
  int32_t* s_j = reinterpret_cast<int32_t*>(smem + RED_BYTES + NODE_BYTES);
  C* s_r = reinterpret_cast<C*>(smem + RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * (cv.cap + 1)));
  const int b = cv.wall_idx[w];
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int vk0 = PH ? cv.vk0 : 0;
  if (PH != 2 && threadIdx.x < 32) {
    // warp 0 stages the interior neighbours in list order (ballot compaction)
    const int lane = threadIdx.x, m = checked_count(cv.cnt[b], cv.cap, cv.status);
    const int32_t* col = cv.col + (int64_t)b * cv.cap;
    const C* R = reinterpret_cast<const C*>(cv.recon) + (int64_t)b * cv.cap;
    int mi = 0;
    for (int s0 = 0; s0 < m; s0 += 32) {
      const int s = s0 + lane;
      const int j = s < m ? checked_index(col[s], cv.n, b, cv.status) : 0;
      const bool in = s < m && cv.kind[j] == 0;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = mi + __popc(bal & ((1u << lane) - 1u));
        s_j[1 + pos] = j;
        s_r[pos] = R[s];
      }
      mi += __popc(bal);
    }
    if (lane == 0) s_j[0] = mi;
  }
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_v[t] = (C)cv.vnodes[t];
  __syncthreads();
  const int mi = PH != 2 ? s_j[0] : 0;
  const int64_t rowlen = (int64_t)NC * NVp;
  S* f = reinterpret_cast<S*>(cv.f_out);
  S* fb = f + (int64_t)b * rowlen;
  const int8_t* cls = cv.wcls + (int64_t)w * NVp;
  const C* vn = reinterpret_cast<const C*>(cv.wvn) + (int64_t)w * NVp;
  const int kb = cv.kind[b];
  const int mrow = kb == cv.lid_wall ? 1 : (cv.body_wall > 0 && kb == cv.body_wall ? 2 : 0);
  const C* Mw = reinterpret_cast<const C*>(cv.mw) + (int64_t)mrow * NVp;
  const C cT = (C)cv.wall_T;

  // flux[0]: sum |c_n| g over the arriving half; flux[1] (PH 1): sum c_n M_w over the
  // leaving half; part: moment sums of the arriving half (PH 0: of the whole row);
  // unit (PH 1): moment sums of M_w over the leaving half
  C flux[2] = {(C)0, (C)0};
  C part[DIM + 2], unit[DIM + 2];
#pragma unroll
  for (int t = 0; t < DIM + 2; ++t) { part[t] = (C)0; unit[t] = (C)0; }
  if (PH != 2) {
    for (int k = threadIdx.x; k < NV; k += blockDim.x) {
      if (cls[k] == 0) {
        C g[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) g[c] = (C)0;
        for (int s = 0; s < mi; ++s) {
          const S* fj = f + (int64_t)s_j[1 + s] * rowlen;
          const C r = s_r[s];
#pragma unroll
          for (int c = 0; c < NC; ++c) g[c] += r * ld1(fj + (int64_t)c * NVp + k);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) st1(fb + (int64_t)c * NVp + k, g[c]);
        flux[0] += vn[k] * g[0];
        int kk = k + vk0;
        C v2 = (C)0;
        part[0] += g[0];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const C va = s_v[kk % nv];
          kk /= nv;
          part[1 + a] += va * g[0];
          v2 += va * va;
        }
        part[DIM + 1] += v2 * g[0];
        if (NC == 2) part[DIM + 1] += g[NC - 1];
      } else if (PH == 1) {
        const C m0 = Mw[k];
        flux[1] += vn[k] * m0;
        int kk = k + vk0;
        C v2 = (C)0;
        unit[0] += m0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const C va = s_v[kk % nv];
          kk /= nv;
          unit[1 + a] += va * m0;
          v2 += va * va;
        }
        unit[DIM + 1] += v2 * m0;
        if (NC == 2) unit[DIM + 1] += cT * m0;
      }
    }
  }
  if constexpr (PH == 1) {
    double t1[DIM + 4], t2[DIM + 2];
    C v1[DIM + 4];
    v1[0] = flux[0];
    v1[1] = flux[1];
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) v1[2 + q] = part[q];
    block_sum0<DIM + 4, C>(v1, t1, s_red);
    block_sum0<DIM + 2, C>(unit, t2, s_red);
    if (threadIdx.x == 0) {
      double* xw = cv.xs + (int64_t)w * wall_sums<DIM>();
#pragma unroll
      for (int q = 0; q < DIM + 4; ++q) xw[q] = t1[q];
#pragma unroll
      for (int q = 0; q < DIM + 2; ++q) xw[DIM + 4 + q] = t2[q];
    }
    return;
  }
  double rho_w;
  if constexpr (PH == 2) {
    const double* xw = cv.xs + (int64_t)w * wall_sums<DIM>();
    rho_w = xw[0] / xw[1];
  } else {
    double ftot[1];
    const C f1[1] = {flux[0]};
    block_sum0<1, C>(f1, ftot, s_red);
    rho_w = ftot[0] * cv.winv[w];
  }
  const C crw = (C)rho_w;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    if (cls[k] != 0) {
      const C g0 = crw * Mw[k];
      st1(fb + k, g0);
      if (NC == 2) st1(fb + NVp + k, cT * g0);
      if (PH == 0) {
        int kk = k;
        C v2 = (C)0;
        part[0] += g0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const C va = s_v[kk % nv];
          kk /= nv;
          part[1 + a] += va * g0;
          v2 += va * va;
        }
        part[DIM + 1] += v2 * g0;
        if (NC == 2) part[DIM + 1] += cT * g0;
      }
    }
  }
  double tot[DIM + 2];
  if constexpr (PH == 2) {
    const double* xw = cv.xs + (int64_t)w * wall_sums<DIM>();
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) tot[q] = xw[2 + q] + rho_w * xw[DIM + 4 + q];
  } else {
    block_sum0<DIM + 2, C>(part, tot, s_red);
  }
  if (threadIdx.x == 0) {
    double rho, Un[3] = {0, 0, 0}, T;
    const double wv = cv.wv;
    finish_moments<DIM>(tot, wv, &rho, Un, &T);
    double* mo = cv.mom + (int64_t)b * MOM_STRIDE;
    mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
    if (!(rho_w >= 0.0) || !isfinite(rho_w)) set_status(cv.status, ST_NONFINITE);
  }
}

// FP32/BF16 storage, the whole wall step (PH = 0 of walls_point): each thread takes 4
// consecutive velocities, so a neighbour row costs one 16-byte (8-byte for BF16) load
// per channel instead of four; the leaving half of the loaded values is unused.  The
// arithmetic per velocity is that of walls_point, with FP32 block sums finished in FP64.
template <typename S, int DIM>
__device__ __forceinline__ void walls_point_v4(const CaseView& cv, const int w, unsigned char* smem) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  double* s_red = reinterpret_cast<double*>(smem);
  float* s_v = reinterpret_cast<float*>(smem + RED_BYTES);
  int32_t* s_j = reinterpret_cast<int32_t*>(smem + RED_BYTES + NODE_BYTES);
  float* s_r = reinterpret_cast<float*>(smem + RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * (cv.cap + 1)));
  const int b = cv.wall_idx[w];
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, m = checked_count(cv.cnt[b], cv.cap, cv.status);
    const int32_t* col = cv.col + (int64_t)b * cv.cap;
    const float* R = reinterpret_cast<const float*>(cv.recon) + (int64_t)b * cv.cap;
    int mi = 0;
    for (int s0 = 0; s0 < m; s0 += 32) {
      const int s = s0 + lane;
      const int j = s < m ? checked_index(col[s], cv.n, b, cv.status) : 0;
      const bool in = s < m && cv.kind[j] == 0;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = mi + __popc(bal & ((1u << lane) - 1u));
        s_j[1 + pos] = j;
        s_r[pos] = R[s];
      }
      mi += __popc(bal);
    }
    if (lane == 0) s_j[0] = mi;
  }
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_v[t] = cv.vnodes_f[t];
  __syncthreads();
  const int mi = s_j[0];
  const int64_t rowlen = (int64_t)NC * NVp;
  S* f = reinterpret_cast<S*>(cv.f_out);
  S* fb = f + (int64_t)b * rowlen;
  const int8_t* cls = cv.wcls + (int64_t)w * NVp;
  const float* vn = reinterpret_cast<const float*>(cv.wvn) + (int64_t)w * NVp;
  const int kb = cv.kind[b];
  const int mrow = kb == cv.lid_wall ? 1 : (cv.body_wall > 0 && kb == cv.body_wall ? 2 : 0);
  const float* Mw = reinterpret_cast<const float*>(cv.mw) + (int64_t)mrow * NVp;
  const float cT = (float)cv.wall_T;
  const int nchunk = NVp >> 2;

  float flux[1] = {0.0f};
  float part[DIM + 2];
#pragma unroll
  for (int t = 0; t < DIM + 2; ++t) part[t] = 0.0f;
  for (int ch = threadIdx.x; ch < nchunk; ch += blockDim.x) {
    const int k0 = 4 * ch;
    const char4 c4 = *reinterpret_cast<const char4*>(cls + k0);
    const bool arr[4] = {c4.x == 0 && k0 < NV, c4.y == 0 && k0 + 1 < NV, c4.z == 0 && k0 + 2 < NV,
                         c4.w == 0 && k0 + 3 < NV};
    if (!(arr[0] || arr[1] || arr[2] || arr[3])) continue;
    float g[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) g[c][e] = 0.0f;
    for (int s = 0; s < mi; ++s) {
      const S* fj = f + (int64_t)s_j[1 + s] * rowlen + k0;
      const float r = s_r[s];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float v[4];
        ld4(fj + (int64_t)c * NVp, v);
#pragma unroll
        for (int e = 0; e < 4; ++e) g[c][e] += r * v[e];
      }
    }
    const float4 vn4 = *reinterpret_cast<const float4*>(vn + k0);
    const float vnv[4] = {vn4.x, vn4.y, vn4.z, vn4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!arr[e]) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) st1(fb + (int64_t)c * NVp + k0 + e, g[c][e]);
      flux[0] += vnv[e] * g[0][e];
      int kk = k0 + e;
      float v2 = 0.0f;
      part[0] += g[0][e];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float va = s_v[kk % nv];
        kk /= nv;
        part[1 + a] += va * g[0][e];
        v2 += va * va;
      }
      part[DIM + 1] += v2 * g[0][e];
      if (NC == 2) part[DIM + 1] += g[NC - 1][e];
    }
  }
  double ftot[1];
  block_sum0<1, float>(flux, ftot, s_red);
  const double rho_w = ftot[0] * cv.winv[w];
  const float crw = (float)rho_w;
  for (int ch = threadIdx.x; ch < nchunk; ch += blockDim.x) {
    const int k0 = 4 * ch;
    const char4 c4 = *reinterpret_cast<const char4*>(cls + k0);
    const bool lv[4] = {c4.x != 0, c4.y != 0, c4.z != 0, c4.w != 0};
    if (!(lv[0] || lv[1] || lv[2] || lv[3])) continue;
    const float4 m4 = *reinterpret_cast<const float4*>(Mw + k0);
    const float mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!lv[e]) continue;
      const float g0 = crw * mw[e];
      st1(fb + k0 + e, g0);
      if (NC == 2) st1(fb + NVp + k0 + e, cT * g0);
      int kk = k0 + e;
      float v2 = 0.0f;
      part[0] += g0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float va = s_v[kk % nv];
        kk /= nv;
        part[1 + a] += va * g0;
        v2 += va * va;
      }
      part[DIM + 1] += v2 * g0;
      if (NC == 2) part[DIM + 1] += cT * g0;
    }
  }
  double tot[DIM + 2];
  block_sum0<DIM + 2, float>(part, tot, s_red);
  if (threadIdx.x == 0) {
    double rho, Un[3] = {0, 0, 0}, T;
    const double wv = cv.wv;
    finish_moments<DIM>(tot, wv, &rho, Un, &T);
    double* mo = cv.mom + (int64_t)b * MOM_STRIDE;
    mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
    if (!(rho_w >= 0.0) || !isfinite(rho_w)) set_status(cv.status, ST_NONFINITE);
  }
}

template <typename S, int DIM>
__global__ void __launch_bounds__(256) k_walls_v4(const CaseView cv) {
  extern __shared__ __align__(16) unsigned char smem[];
  walls_point_v4<S, DIM>(cv, blockIdx.x, smem);
}

template <typename S, typename C, int DIM, int PH = 0>
__global__ void __launch_bounds__(256) k_walls(const CaseView cv) {
  extern __shared__ __align__(16) unsigned char smem[];
  walls_point<S, C, DIM, PH>(cv, blockIdx.x, smem);
}

// witems[k] = (case, wall slot): one CTA per wall point of any case (2D: the body of
// k_walls, so that batched and per-case stepping give the same bits)
template <typename S, typename C, int DIM>
__global__ void __launch_bounds__(256) k_walls_batch(const CaseView* __restrict__ cases, const int2* __restrict__ witems) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int2 e = witems[blockIdx.x];
  walls_point<S, C, DIM>(cases[e.x], e.y, smem);
}

int launch_transport_batch(const CaseView* d_cases, const int2* items, int n_items, int dim, int storage, int capmax,
                           int warps, int grid, cudaStream_t s) {
  if (n_items == 0) return 0;
  const int threads = 32 * warps;
  const size_t smem = dim == 2 ? wp_smem_bytes<2>(warps, capmax) : wp_smem_bytes<3>(warps, capmax);
  const int ntiles = (n_items + warps - 1) / warps;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
#define BGK_BATCH(S, D)                                                                    \
  {                                                                                        \
    auto k = k_transport_batch<S, D>;                                                      \
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    k<<<grid, threads, smem, s>>>(d_cases, items, n_items, capmax);                        \
  }
  if (dim == 2) {
    if (storage == 1) BGK_BATCH(float, 2) else BGK_BATCH(__nv_bfloat16, 2)
  } else {
    if (storage == 1) BGK_BATCH(float, 3) else BGK_BATCH(__nv_bfloat16, 3)
  }
#undef BGK_BATCH
  return 1;
}

int launch_walls_batch(const CaseView* d_cases, const int2* witems, int n_witems, int dim, int storage, int capmax,
                       cudaStream_t s) {
  if (n_witems == 0) return 0;
  const size_t smem = RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * (capmax + 1)) + sizeof(double) * capmax;
  if (dim == 2) {
    if (storage == 1) k_walls_batch<float, float, 2><<<n_witems, 256, smem, s>>>(d_cases, witems);
    else k_walls_batch<__nv_bfloat16, float, 2><<<n_witems, 256, smem, s>>>(d_cases, witems);
  } else {
    if (storage == 1) k_walls_batch<float, float, 3><<<n_witems, 256, smem, s>>>(d_cases, witems);
    else k_walls_batch<__nv_bfloat16, float, 3><<<n_witems, 256, smem, s>>>(d_cases, witems);
  }
  return 1;
}

int launch_walls(const CaseView& cv, cudaStream_t s) {
  if (cv.n_wall == 0) return 0;
  const int threads = 256;
  const size_t smem = RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * (cv.cap + 1)) + sizeof(double) * cv.cap;
  // 2D keeps the one-velocity-per-thread body: beside the side-chain kernel of an ALE step
  // the vector body's extra registers (43 against 32) slow the chain more than they save
  // (201^2 x 32^2 ALE cavity: 0.4925 against 0.4857 ms per step, chain 61 against 53 us);
  // in 3D, with no side chain, the vector body wins (41^3 x 16^3: 6.45 against 6.63 ms).
  if (cv.dim == 2) {
    if (cv.storage == 0) k_walls<double, double, 2><<<cv.n_wall, threads, smem, s>>>(cv);
    else if (cv.storage == 1) k_walls<float, float, 2><<<cv.n_wall, threads, smem, s>>>(cv);
    else k_walls<__nv_bfloat16, float, 2><<<cv.n_wall, threads, smem, s>>>(cv);
  } else {
    if (cv.storage == 0) k_walls<double, double, 3><<<cv.n_wall, threads, smem, s>>>(cv);
    else if (cv.storage == 1) k_walls_v4<float, 3><<<cv.n_wall, threads, smem, s>>>(cv);
    else k_walls_v4<__nv_bfloat16, 3><<<cv.n_wall, threads, smem, s>>>(cv);
  }
  return 1;
}

// ---------------------------------------------------------------------------
// wall tables: classification by the normal velocity relative to the wall,
// c_n = (v - u_w).n, |c_n|, 1/sum_{c_n>0} c_n M_w and the unit-density wall
// Maxwellians, all evaluated in FP64.  u_w is lid_u on the lid, body_u on the
// body, zero elsewhere; the tables stay valid while the walls translate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ const double* wall_velocity(const CaseView& cv, int kb, const double* zero) {
  if (kb == cv.lid_wall) return cv.lid_u;
  if (cv.body_wall > 0 && kb == cv.body_wall) return cv.body_u;
  return zero;
}

template <typename C, int DIM>
__global__ void k_wall_tables(CaseView cv) {
  __shared__ double s_sum[32];
  const int w = blockIdx.x;
  const int b = cv.wall_idx[w];
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  double nb[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) nb[a] = cv.normal[(int64_t)b * DIM + a];
  const double zero[3] = {0.0, 0.0, 0.0};
  const double* uw = wall_velocity(cv, cv.kind[b], zero);
  const double pi = 3.14159265358979323846, T = cv.wall_T;
  const double pref = DIM == 2 ? 1.0 / (2.0 * pi * T) : 1.0 / pow(2.0 * pi * T, 1.5);
  double acc = 0.0;
  for (int k = threadIdx.x; k < NVp; k += blockDim.x) {
    int8_t cl = 0;
    double avn = 0.0;
    if (k < NV) {
      int kk = k + cv.vk0;
      double vn = 0.0, c2 = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double va = cv.vnodes[kk % nv];
        kk /= nv;
        const double c = __dadd_rn(va, -uw[a]);
        vn = __dadd_rn(vn, __dmul_rn(c, nb[a]));
        c2 += c * c;
      }
      cl = vn > 0.0 ? 1 : 0;
      avn = fabs(vn);
      if (cl) acc += vn * (pref * exp(-c2 / (2.0 * T)));
    }
    cv.wcls[(int64_t)w * NVp + k] = cl;
    reinterpret_cast<C*>(cv.wvn)[(int64_t)w * NVp + k] = (C)avn;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) s += s_sum[q];
    // a velocity slab of a sharded case holds part of this sum (its wall step takes
    // the sum over all slabs instead): no check there
    const bool slab = cv.vk0 != 0 || NV != (DIM == 2 ? nv * nv : nv * nv * nv);
    cv.winv[w] = s > 0.0 ? 1.0 / s : 0.0;
    if (!(s > 0.0) && !slab) set_status(cv.status, ST_SINGULAR);
  }
}

template <typename C, int DIM>
__global__ void k_mw_table(CaseView cv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cv.NVp) return;
  const double pi = 3.14159265358979323846, T = cv.wall_T;
  const double pref = DIM == 2 ? 1.0 / (2.0 * pi * T) : 1.0 / pow(2.0 * pi * T, 1.5);
  const double zero[3] = {0.0, 0.0, 0.0};
  for (int row = 0; row < 3; ++row) {
    const double* uw = row == 0 ? zero : (row == 1 ? cv.lid_u : cv.body_u);
    double M = 0.0;
    if (k < cv.NV) {
      int kk = k + cv.vk0;
      double c2 = 0.0;
      for (int a = 0; a < DIM; ++a) {
        const double c = cv.vnodes[kk % cv.nv] - uw[a];
        kk /= cv.nv;
        c2 += c * c;
      }
      M = pref * exp(-c2 / (2.0 * T));
    }
    reinterpret_cast<C*>(cv.mw)[row * cv.NVp + k] = (C)M;
  }
}

// Velocity nodes v_j = -vmax + j dv in the centred form (j - (nv-1)/2) dv, exactly
// symmetric about zero (Sec. 3.3).
__global__ void k_nodes(CaseView cv) {
  const int j = threadIdx.x;
  if (j < cv.nv) {
    const double v = __dmul_rn(__dadd_rn((double)j, -0.5 * (double)(cv.nv - 1)), cv.dv);
    cv.vnodes[j] = v;
    cv.vnodes_f[j] = (float)v;
  }
}

int launch_init_tables(const CaseView& cv, cudaStream_t s) {
  int n = 1;
  k_nodes<<<1, 64, 0, s>>>(cv);
  const bool f64 = cv.storage == 0;
  if (cv.dim == 2) {
    if (f64) k_mw_table<double, 2><<<grid_for(cv.NVp, 256), 256, 0, s>>>(cv);
    else k_mw_table<float, 2><<<grid_for(cv.NVp, 256), 256, 0, s>>>(cv);
  } else {
    if (f64) k_mw_table<double, 3><<<grid_for(cv.NVp, 256), 256, 0, s>>>(cv);
    else k_mw_table<float, 3><<<grid_for(cv.NVp, 256), 256, 0, s>>>(cv);
  }
  ++n;
  if (cv.n_wall > 0) {
    if (cv.dim == 2) {
      if (f64) k_wall_tables<double, 2><<<cv.n_wall, 256, 0, s>>>(cv);
      else k_wall_tables<float, 2><<<cv.n_wall, 256, 0, s>>>(cv);
    } else {
      if (f64) k_wall_tables<double, 3><<<cv.n_wall, 256, 0, s>>>(cv);
      else k_wall_tables<float, 3><<<cv.n_wall, 256, 0, s>>>(cv);
    }
    ++n;
  }
  return n;
}

// ---------------------------------------------------------------------------
// point motion (Eqs. originalALE1, ALE1)
// ---------------------------------------------------------------------------
// After every CTA has read the body centre and merged its maximum squared
// displacement (bits b) into disp2, the last one decides whether the next list
// build rebuilds the candidates and advances the centre to cn.
__device__ __forceinline__ void move_merge(const CaseView& cv, uint32_t b, double thr2, const double* cn) {
  if (cv.sk) atomicMax(&cv.sk->disp2, b);
  __threadfence();
  uint32_t* ctr = cv.sk ? &cv.sk->blocks : &cv.body->blocks;
  if (atomicAdd(ctr, 1u) == gridDim.x - 1) {
    __threadfence();
    if (cv.sk) {
      const uint32_t d = atomicOr(&cv.sk->disp2, 0u);
      const int rb = (double)__uint_as_float(d) > thr2;
      cv.sk->rebuild = rb;
      if (rb) cv.sk->disp2 = 0u;
    }
    if (cv.body)
      for (int a = 0; a < cv.dim; ++a) cv.body->c[a] = cn[a];
    *ctr = 0u;
  }
}

// Threads [0, n_int) move the interior points, threads [n_int, n_int + n_wall) the
// body's boundary points among the wall points (when there is a body).  With skin
// lists the kernel also tracks max |x - x_b|^2; its last CTA decides whether the next
// list build rebuilds the candidates (max |x - x_b| > h skin / 2, thr2 = (h skin /
// 2)^2 (1 - 1e-6)) and advances the body centre.
__global__ void __launch_bounds__(256) k_move(CaseView cv, double thr2) {
  __shared__ uint32_t s_max[8];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double cn[3];
  body_centre_next(cv, cn);
  const double d2 = move_thread(cv, t, cn);
  if (cv.sk || cv.body) {
    // CTA maximum of the displacement bits (non-negative floats order as integers)
    const uint32_t w = __reduce_max_sync(0xffffffffu, __float_as_uint(__double2float_ru(d2)));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t b = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b = max(b, s_max[k]);
      move_merge(cv, b, thr2, cn);
    }
  }
}

int launch_move(const CaseView& cv, cudaStream_t s) {
  const int64_t n = (int64_t)cv.n_int + (cv.body ? cv.n_wall : 0);
  if (n == 0) return 0;
  const double half = 0.5 * cv.h * cv.skin;
  k_move<<<grid_for(n, 256), 256, 0, s>>>(cv, half * half * (1.0 - 1e-6));
  return 1;
}

// ---------------------------------------------------------------------------
// initial Maxwellian, moments of a given f, layout conversion
// ---------------------------------------------------------------------------
// The same Maxwellian at every point: thread k of column block y evaluates M(v_k) once and
// writes it (and T0 M, the Chu h component) into the rows of the points of its block
// (blockIdx.x, blockIdx.x + gridDim.x, ...), so that a grid of a few hundred blocks
// evaluates a few hundred rows' worth of exponentials, not one per (point, velocity).
template <typename S, int DIM>
__global__ void k_set_maxwellian(CaseView cv, double rho0, double u0, double u1, double u2, double T0) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= cv.NVp) return;
  const double pi = 3.14159265358979323846;
  double M = 0.0;
  if (k < cv.NV) {
    const double U[3] = {u0, u1, u2};
    int kk = k + cv.vk0;
    double c2 = 0.0;
    for (int a = 0; a < DIM; ++a) {
      const double c = cv.vnodes[kk % cv.nv] - U[a];
      kk /= cv.nv;
      c2 += c * c;
    }
    const double pref = DIM == 2 ? rho0 / (2.0 * pi * T0) : rho0 / pow(2.0 * pi * T0, 1.5);
    M = pref * exp(-c2 / (2.0 * T0));
  }
  using C = decltype(ld1(reinterpret_cast<const S*>(cv.f_in)));
  const C m0 = (C)M, m1 = (C)(T0 * M);
  for (int i = blockIdx.x; i < cv.n; i += gridDim.x) {
    S* f = reinterpret_cast<S*>(cv.f_in) + (int64_t)i * NC * cv.NVp;
    st1(f + k, m0);
    if (NC == 2) st1(f + cv.NVp + k, m1);
  }
}

int launch_set_maxwellian(const CaseView& cv, double rho0, const double* u0, double T0, cudaStream_t s) {
  const dim3 g((unsigned)std::min(cv.n, 1216), (unsigned)((cv.NVp + 255) / 256));
  if (cv.dim == 2) {
    if (cv.storage == 0) k_set_maxwellian<double, 2><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], 0.0, T0);
    else if (cv.storage == 1) k_set_maxwellian<float, 2><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], 0.0, T0);
    else k_set_maxwellian<__nv_bfloat16, 2><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], 0.0, T0);
  } else {
    if (cv.storage == 0) k_set_maxwellian<double, 3><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], u0[2], T0);
    else if (cv.storage == 1) k_set_maxwellian<float, 3><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], u0[2], T0);
    else k_set_maxwellian<__nv_bfloat16, 3><<<g, 256, 0, s>>>(cv, rho0, u0[0], u0[1], u0[2], T0);
  }
  return 1;
}

// Moments of every point of f (internal layout), one CTA per point.  SH: the raw sums
// of the velocity slab to the exchange buffer instead.
template <typename S, typename C, int DIM, bool SH = false>
__global__ void k_moments(CaseView cv, const S* f) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  __shared__ double s_red[8 * 32];
  const int i = blockIdx.x;
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const S* fi = f + (int64_t)i * NC * NVp;
  C part[DIM + 2];
#pragma unroll
  for (int t = 0; t < DIM + 2; ++t) part[t] = (C)0;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    const C g = ld1(fi + k);
    int kk = k + (SH ? cv.vk0 : 0);
    C v2 = (C)0;
    part[0] += g;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const C va = (C)cv.vnodes[kk % nv];
      kk /= nv;
      part[1 + a] += va * g;
      v2 += va * va;
    }
    part[DIM + 1] += v2 * g;
    if (NC == 2) part[DIM + 1] += ld1(fi + NVp + k);
  }
  double tot[DIM + 2];
  block_sum0<DIM + 2, C>(part, tot, s_red);
  if (SH && threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) cv.xs[(int64_t)i * (DIM + 2) + q] = tot[q];
  } else if (threadIdx.x == 0) {
    double rho, Un[3] = {0, 0, 0}, T;
    const double wv = cv.wv;
    finish_moments<DIM>(tot, wv, &rho, Un, &T);
    double* mo = cv.mom + (int64_t)i * MOM_STRIDE;
    mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
  }
}

// FP32/BF16 storage: each warp streams MOM_GP consecutive points in turn, each lane 4
// consecutive velocities per chunk (16-byte loads, eight chunks in flight, velocity nodes
// staged in shared memory as FP32) into Kahan-compensated FP32 sums.  A point's lane sums
// are reduced across the warp as FP32 pairs with exact high-part additions (no FP64 on
// the 32-lane path); once the warp has all its points, lane g converts point g's pair
// totals to FP64 and forms rho, U, T in FP64, so each FP64 instruction serves MOM_GP
// points (FP64 runs at a small fraction of the FP32 rate).  SH: the raw sums of the
// velocity slab (in FP64) to the exchange buffer instead.
constexpr int MOM_GP = 8, MOM_WARPS = 4;  // points per warp, warps per CTA
template <typename S, int DIM, bool ROW, bool SH = false>
__global__ void __launch_bounds__(32 * MOM_WARPS) k_moments_wp(CaseView cv, const S* f) {
  constexpr int NC = DIM == 2 ? 2 : 1, VPL = 4, NQ = DIM + 2;
  __shared__ __align__(16) float s_v[64];  // chunk_velocities reads groups of 4
  __shared__ float2 s_tot[MOM_WARPS][MOM_GP][NQ];
  for (int t = threadIdx.x; t < cv.nv; t += blockDim.x) s_v[t] = cv.vnodes_f[t];
  __syncthreads();
  const int W = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (blockIdx.x * W + warp) * MOM_GP;
  if (i0 >= cv.n) return;
  const int np = min(MOM_GP, cv.n - i0);
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int vk0 = SH ? cv.vk0 : 0;
  const float inv_nv = 1.0f / (float)nv;
  for (int g = 0; g < np; ++g) {
    const S* fi = f + (int64_t)(i0 + g) * NC * NVp;
    float msum[NQ], mcmp[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { msum[q] = 0.0f; mcmp[q] = 0.0f; }
#pragma unroll 8
    for (int chunk = lane; chunk * VPL < NVp; chunk += 32) {
      const int k0 = chunk * VPL;
      float vel[VPL][DIM];
      bool kin[VPL];
      chunk_velocities<DIM, VPL, ROW>(k0 + vk0, nv, NV + vk0, inv_nv, s_v, vel, kin);
      float gv[NC][VPL];
#pragma unroll
      for (int c = 0; c < NC; ++c) ldv<S, VPL>(fi + (int64_t)c * NVp + k0, gv[c]);
      float ps[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) ps[q] = 0.0f;
#pragma unroll
      for (int e = 0; e < VPL; ++e) {
        const float g0 = kin[e] ? gv[0][e] : 0.0f;
        float v2 = 0.0f;
        ps[0] += g0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) { ps[1 + a] = fmaf(vel[e][a], g0, ps[1 + a]); v2 = fmaf(vel[e][a], vel[e][a], v2); }
        ps[DIM + 1] = fmaf(v2, g0, ps[DIM + 1]);
        if (NC == 2) ps[DIM + 1] += kin[e] ? gv[NC - 1][e] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float y = ps[q] - mcmp[q];
        const float t = msum[q] + y;
        mcmp[q] = (t - msum[q]) - y;
        msum[q] = t;
      }
    }
    // warp totals as FP32 pairs (every lane ends with the same pair)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float hi = msum[q], lo = -mcmp[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        pair_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
      if (lane == 0) s_tot[warp][g][q] = make_float2(hi, lo);
    }
  }
  __syncwarp();
  if (lane >= np) return;
  const int i = i0 + lane;
  double tot[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) tot[q] = (double)s_tot[warp][lane][q].x + (double)s_tot[warp][lane][q].y;
  if (SH) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) cv.xs[(int64_t)i * NQ + q] = tot[q];
  } else {
    double rho, Un[3] = {0, 0, 0}, T;
    const double wv = cv.wv;
    finish_moments<DIM>(tot, wv, &rho, Un, &T);
    double* mo = cv.mom + (int64_t)i * MOM_STRIDE;
    mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
  }
}

int launch_moments(const CaseView& cv, const void* f, cudaStream_t s) {
  const int W = MOM_WARPS, grid = (cv.n + W * MOM_GP - 1) / (W * MOM_GP);
  const bool row = cv.nv % 4 == 0;
#define BGK_MOM_WP(S, D)                                                                               \
  {                                                                                                    \
    if (row) k_moments_wp<S, D, true><<<grid, 32 * W, 0, s>>>(cv, (const S*)f);                        \
    else k_moments_wp<S, D, false><<<grid, 32 * W, 0, s>>>(cv, (const S*)f);                           \
  }
  if (cv.dim == 2) {
    if (cv.storage == 0) k_moments<double, double, 2><<<cv.n, 256, 0, s>>>(cv, (const double*)f);
    else if (cv.storage == 1) BGK_MOM_WP(float, 2)
    else BGK_MOM_WP(__nv_bfloat16, 2)
  } else {
    if (cv.storage == 0) k_moments<double, double, 3><<<cv.n, 256, 0, s>>>(cv, (const double*)f);
    else if (cv.storage == 1) BGK_MOM_WP(float, 3)
    else BGK_MOM_WP(__nv_bfloat16, 3)
  }
#undef BGK_MOM_WP
  return 1;
}

// ---------------------------------------------------------------------------
// velocity-sharded step: slabs of the velocity grid, each advanced by the kernels
// above with its velocity offset; the slabs couple only through the sums in cv.xs
// ---------------------------------------------------------------------------
template <typename S, int DIM>
static void launch_shard_transport_wp(const CaseView& cv, cudaStream_t s) {
  const int W = BGK_WP_WARPS, threads = 32 * W;
  const size_t smem = wp_smem_bytes<DIM>(W, cv.cap);
  const int grid = (cv.n_int + W - 1) / W;
  const bool row4 = cv.nv % 4 == 0;
#define BGK_LAUNCH_SH(ALE, ROW)                                                           \
  {                                                                                       \
    auto k = k_transport_wp<S, DIM, ALE, ROW, 4, true>;                                   \
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    k<<<grid, threads, smem, s>>>(cv);                                                    \
  }
  if (cv.ale) {
    if (row4) BGK_LAUNCH_SH(true, true) else BGK_LAUNCH_SH(true, false)
  } else {
    if (row4) BGK_LAUNCH_SH(false, true) else BGK_LAUNCH_SH(false, false)
  }
#undef BGK_LAUNCH_SH
}

int launch_shard_transport(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) launch_transport_d<double, double, 2, true>(cv, s);
    else if (cv.storage == 1) launch_shard_transport_wp<float, 2>(cv, s);
    else launch_shard_transport_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 0) launch_transport_d<double, double, 3, true>(cv, s);
    else if (cv.storage == 1) launch_shard_transport_wp<float, 3>(cv, s);
    else launch_shard_transport_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

template <typename S, int DIM>
static void launch_shard_relax_wp(const CaseView& cv, cudaStream_t s) {
  const int W = 8, grid = (cv.n_int + W - 1) / W;
  if (cv.nv % 4 == 0) k_shard_relax_wp<S, DIM, true><<<grid, 32 * W, 0, s>>>(cv);
  else k_shard_relax_wp<S, DIM, false><<<grid, 32 * W, 0, s>>>(cv);
}

int launch_shard_relax(const CaseView& cv, cudaStream_t s) {
  if (cv.n_int == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) launch_shard_relax_d<double, double, 2>(cv, s);
    else if (cv.storage == 1) launch_shard_relax_wp<float, 2>(cv, s);
    else launch_shard_relax_wp<__nv_bfloat16, 2>(cv, s);
  } else {
    if (cv.storage == 0) launch_shard_relax_d<double, double, 3>(cv, s);
    else if (cv.storage == 1) launch_shard_relax_wp<float, 3>(cv, s);
    else launch_shard_relax_wp<__nv_bfloat16, 3>(cv, s);
  }
  return 1;
}

int launch_shard_walls(const CaseView& cv, int phase, cudaStream_t s) {
  if (cv.n_wall == 0) return 0;
  const size_t smem = RED_BYTES + NODE_BYTES + align16(sizeof(int32_t) * (cv.cap + 1)) + sizeof(double) * cv.cap;
#define BGK_WALLS_PH(S, C, D)                                                          \
  {                                                                                    \
    if (phase == 1) k_walls<S, C, D, 1><<<cv.n_wall, 256, smem, s>>>(cv);              \
    else k_walls<S, C, D, 2><<<cv.n_wall, 256, smem, s>>>(cv);                         \
  }
  if (cv.dim == 2) {
    if (cv.storage == 0) BGK_WALLS_PH(double, double, 2)
    else if (cv.storage == 1) BGK_WALLS_PH(float, float, 2)
    else BGK_WALLS_PH(__nv_bfloat16, float, 2)
  } else {
    if (cv.storage == 0) BGK_WALLS_PH(double, double, 3)
    else if (cv.storage == 1) BGK_WALLS_PH(float, float, 3)
    else BGK_WALLS_PH(__nv_bfloat16, float, 3)
  }
#undef BGK_WALLS_PH
  return 1;
}

int launch_shard_partial(const CaseView& cv, cudaStream_t s) {
  const int W = MOM_WARPS, grid = (cv.n + W * MOM_GP - 1) / (W * MOM_GP);
  const bool row = cv.nv % 4 == 0;
#define BGK_PART_WP(S, D)                                                                                   \
  {                                                                                                         \
    if (row) k_moments_wp<S, D, true, true><<<grid, 32 * W, 0, s>>>(cv, (const S*)cv.f_in);                 \
    else k_moments_wp<S, D, false, true><<<grid, 32 * W, 0, s>>>(cv, (const S*)cv.f_in);                    \
  }
  if (cv.dim == 2) {
    if (cv.storage == 0) k_moments<double, double, 2, true><<<cv.n, 256, 0, s>>>(cv, (const double*)cv.f_in);
    else if (cv.storage == 1) BGK_PART_WP(float, 2)
    else BGK_PART_WP(__nv_bfloat16, 2)
  } else {
    if (cv.storage == 0) k_moments<double, double, 3, true><<<cv.n, 256, 0, s>>>(cv, (const double*)cv.f_in);
    else if (cv.storage == 1) BGK_PART_WP(float, 3)
    else BGK_PART_WP(__nv_bfloat16, 3)
  }
#undef BGK_PART_WP
  return 1;
}

template <int DIM>
__global__ void k_shard_moments(CaseView cv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  double tot[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) tot[q] = cv.xs[(int64_t)i * (DIM + 2) + q];
  double rho, Un[3] = {0, 0, 0}, T;
  const double wv = cv.wv;
  finish_moments<DIM>(tot, wv, &rho, Un, &T);
  double* mo = cv.mom + (int64_t)i * MOM_STRIDE;
  mo[0] = rho; mo[1] = Un[0]; mo[2] = Un[1]; mo[3] = Un[2]; mo[4] = T;
}

int launch_shard_moments(const CaseView& cv, cudaStream_t s) {
  if (cv.dim == 2) k_shard_moments<2><<<grid_for(cv.n, 256), 256, 0, s>>>(cv);
  else k_shard_moments<3><<<grid_for(cv.n, 256), 256, 0, s>>>(cv);
  return 1;
}

// One-device stand-in for the allreduce of the slabs' sums: every element is summed
// over the buffers in buffer order and the sum is written to every buffer, so that
// all slabs continue from the same bits.
struct ShardBufs {
  double* p[SHARD_MAX_BUFS];
};

__global__ void k_shard_allreduce(ShardBufs b, int nb, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int r = 0; r < nb; ++r) sum += b.p[r][e];
    for (int r = 0; r < nb; ++r) b.p[r][e] = sum;
  }
}

int launch_shard_allreduce(double* const* bufs, int nbufs, int64_t count, cudaStream_t s) {
  if (count <= 0) return 0;
  ShardBufs b;
  for (int r = 0; r < SHARD_MAX_BUFS; ++r) b.p[r] = r < nbufs ? bufs[r] : nullptr;
  const int64_t blocks = (count + 255) / 256;
  k_shard_allreduce<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(b, nbufs, count);
  return 1;
}

template <typename A, typename B>
__global__ void k_pack(const A* src, B* dst, int64_t rows, int NV, int NVp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * NVp) return;
  const int64_t r = t / NVp;
  const int k = (int)(t % NVp);
  const float fz = 0.0f;
  if (k < NV) st1(dst + t, (decltype(ld1(dst)))ld1(src + r * NV + k));
  else st1(dst + t, (decltype(ld1(dst)))fz);
}

template <typename A, typename B>
__global__ void k_unpack(const A* src, B* dst, int64_t rows, int NV, int NVp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * NV) return;
  const int64_t r = t / NV;
  const int k = (int)(t % NV);
  st1(dst + t, (decltype(ld1(dst)))ld1(src + r * NVp + k));
}

template <typename A>
static void pack_from(const CaseView& cv, const A* src, void* dst, cudaStream_t s) {
  const int64_t rows = (int64_t)cv.n * cv.ncomp;
  const int g = (int)((rows * cv.NVp + 255) / 256);
  if (cv.storage == 0) k_pack<A, double><<<g, 256, 0, s>>>(src, (double*)dst, rows, cv.NV, cv.NVp);
  else if (cv.storage == 1) k_pack<A, float><<<g, 256, 0, s>>>(src, (float*)dst, rows, cv.NV, cv.NVp);
  else k_pack<A, __nv_bfloat16><<<g, 256, 0, s>>>(src, (__nv_bfloat16*)dst, rows, cv.NV, cv.NVp);
}

template <typename B>
static void unpack_to(const CaseView& cv, const void* src, B* dst, cudaStream_t s) {
  const int64_t rows = (int64_t)cv.n * cv.ncomp;
  const int g = (int)((rows * cv.NV + 255) / 256);
  if (cv.storage == 0) k_unpack<double, B><<<g, 256, 0, s>>>((const double*)src, dst, rows, cv.NV, cv.NVp);
  else if (cv.storage == 1) k_unpack<float, B><<<g, 256, 0, s>>>((const float*)src, dst, rows, cv.NV, cv.NVp);
  else k_unpack<__nv_bfloat16, B><<<g, 256, 0, s>>>((const __nv_bfloat16*)src, dst, rows, cv.NV, cv.NVp);
}

int launch_pack_f(const CaseView& cv, const void* src, int src_dtype, void* dst, cudaStream_t s) {
  if (src_dtype == 0) pack_from(cv, (const double*)src, dst, s);
  else if (src_dtype == 1) pack_from(cv, (const float*)src, dst, s);
  else pack_from(cv, (const __nv_bfloat16*)src, dst, s);
  return 1;
}

int launch_unpack_f(const CaseView& cv, const void* src, void* dst, int dst_dtype, cudaStream_t s) {
  if (dst_dtype == 0) unpack_to(cv, src, (double*)dst, s);
  else if (dst_dtype == 1) unpack_to(cv, src, (float*)dst, s);
  else unpack_to(cv, src, (__nv_bfloat16*)dst, s);
  return 1;
}

}  // namespace bgk
