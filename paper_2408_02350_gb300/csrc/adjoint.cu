// Discrete adjoint of one time step (fixed points) and the lid-flux objective.
//
// The step map f^{n+1} = Phi(f^n; u_lid, Kn) of the forward kernels is
//   f~ = L f            positive upwind transport, linear for fixed points
//   y  = a f~ + b M     relaxation, (rho, U, T) = moments(f~), a = tau/(tau+dt), b = 1 - a
//   f^{n+1} = [y at interior points; W(y) at wall points]
// with W the WLS reconstruction of arriving velocities and rho_w M_w on leaving
// ones, rho_w = F / N (F the arriving normal mass flux, N the normalisation of
// the unit-density wall Maxwellian, which depends on u_lid).  Given the state
// f^n and lam1 = dJ/df^{n+1}, one adjoint step computes lam0 = (dPhi/df^n)^T lam1
// and adds dJ/du_lid and dJ/dKn to a device accumulator, in four kernels:
//   k_adj_prep       recompute f~ and y from f^n (interior points)
//   k_adj_walls      per wall point: mu = dJ/drho_w and the lid-velocity derivative
//   k_adj_relax      per interior point: lam_y = lam1 + wall terms, then the VJP of
//                    the relaxation through rho, U, T, tau and M (Kn derivative)
//   k_adj_transport  lam0 = L^T lam_f~ as a gather: the neighbour relation is
//                    symmetric, and tslot[p][t] is the slot of p in the row of its
//                    t-th neighbour, so each point sums its own contributions.
#include <cuda_runtime.h>

#include "bgk_internal.cuh"
#include "device_common.cuh"

namespace bgk {

namespace {
constexpr int RED = 16 * 32;  // doubles of block-reduction scratch (16 values x 32 warps)

inline int grid_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

template <int NVAL>
__device__ __forceinline__ void block_reduce(double (&v)[NVAL], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NVAL; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) scratch[q * 32 + warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < NVAL) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += scratch[threadIdx.x * 32 + w];
    scratch[threadIdx.x * 32] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NVAL; ++q) v[q] = scratch[q * 32];
  __syncthreads();
}

template <typename C> __device__ __forceinline__ C cmin(C a, C b) { return a < b ? a : b; }
__device__ __forceinline__ float cexp(float x) { return expf(x); }
__device__ __forceinline__ double cexp(double x) { return exp(x); }

// velocity components of node k
template <int DIM>
__device__ __forceinline__ void vel_of(int k, int nv, const double* nodes, double (&v)[DIM]) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) { v[a] = nodes[k % nv]; k /= nv; }
}
}  // namespace

// transpose slot map: tslot[p][t] = position of p in the row of col[p][t] (-1 if absent)
__global__ void k_tslot(CaseView cv, int32_t* tslot) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cv.n) return;
  const int cap = cv.cap, m = cv.cnt[p];
  for (int t = 0; t < m; ++t) {
    const int i = cv.col[(int64_t)p * cap + t];
    const int32_t* row = cv.col + (int64_t)i * cap;
    int lo = 0, hi = cv.cnt[i] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int v = row[mid];
      if (v == p) { pos = mid; break; }
      if (v < p) lo = mid + 1; else hi = mid - 1;
    }
    tslot[(int64_t)p * cap + t] = pos;
  }
}

// f~ and y = relax(f~) at interior points (compute type C, internal layout)
template <typename S, typename C, int DIM>
__global__ void __launch_bounds__(256) k_adj_prep(CaseView cv, C* FT, C* Y) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  __shared__ double s_red[RED];
  __shared__ double s_nodes[64];
  __shared__ double s_fin[8];
  const int i = cv.int_idx[blockIdx.x];
  const int m = cv.cnt[i], cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_nodes[t] = cv.vnodes[t];
  __syncthreads();
  const S* f = reinterpret_cast<const S*>(cv.f_in);
  const C* P = reinterpret_cast<const C*>(cv.P) + (int64_t)i * cap * DD;
  const int32_t* row = cv.col + (int64_t)i * cap;
  const int64_t rowlen = (int64_t)NC * NVp;
  const C two_dt = (C)(2.0 * cv.dt);
  C cpart[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) cpart[q] = (C)0;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C v[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) v[a] = (C)vd[a];
    C acc[NC], sk = (C)0, fi[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { acc[c] = (C)0; fi[c] = ld1(f + (int64_t)i * rowlen + (int64_t)c * NVp + k); }
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      C mk = (C)0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        C pd = (C)0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) pd += v[a] * P[s * DD + d * DIM + a];
        mk += cmin(pd, (C)0);
      }
      sk += mk;
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += mk * ld1(f + (int64_t)j * rowlen + (int64_t)c * NVp + k);
    }
    C v2 = (C)0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const C ft = fi[c] - two_dt * (acc[c] - sk * fi[c]);
      FT[(int64_t)i * rowlen + (int64_t)c * NVp + k] = ft;
      if (c == 0) {
        cpart[0] += ft;
#pragma unroll
        for (int a = 0; a < DIM; ++a) { cpart[1 + a] += v[a] * ft; v2 += v[a] * v[a]; }
        cpart[DIM + 1] += v2 * ft;
      } else {
        cpart[DIM + 1] += ft;
      }
    }
  }
  double part[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) part[q] = (double)cpart[q];
  block_reduce<DIM + 2>(part, s_red);
  if (threadIdx.x == 0) {
    const double R = part[0];
    double U[3] = {0, 0, 0}, u2 = 0.0;
    for (int a = 0; a < DIM; ++a) { U[a] = part[1 + a] / R; u2 += U[a] * U[a]; }
    const double T = (part[DIM + 1] - R * u2) / (3.0 * R);
    const double wv = cv.wv;
    const double rho = R * wv, pi = 3.14159265358979323846;
    double a = 1.0, b = 0.0;
    if (cv.tau_mode != 2) {
      const double tau = cv.tau_mode == 1 ? sqrt(2.0 / pi) * cv.kn : sqrt(2.0 / pi) * cv.kn / (rho * sqrt(T));
      a = tau / (tau + cv.dt);
      b = cv.dt / (tau + cv.dt);
    }
    s_fin[0] = a; s_fin[1] = b; s_fin[2] = rho; s_fin[3] = T;
    for (int q = 0; q < 3; ++q) s_fin[4 + q] = U[q];
  }
  __syncthreads();
  const C a = (C)s_fin[0], b = (C)s_fin[1], T = (C)s_fin[3];
  const double pi = 3.14159265358979323846;
  const C pref = (C)(DIM == 2 ? s_fin[2] / (2.0 * pi * s_fin[3]) : s_fin[2] / pow(2.0 * pi * s_fin[3], 1.5));
  const C nl2 = (C)(-0.5 / s_fin[3]);
  C Uc[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) Uc[d] = (C)s_fin[4 + d];
  for (int k = threadIdx.x; k < NVp; k += blockDim.x) {
    if (k >= NV) {
#pragma unroll
      for (int c = 0; c < NC; ++c) Y[(int64_t)i * rowlen + (int64_t)c * NVp + k] = (C)0;
      continue;
    }
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C c2 = (C)0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) { const C cc = (C)vd[d] - Uc[d]; c2 += cc * cc; }
    const C M0 = pref * cexp(nl2 * c2);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const C ft = FT[(int64_t)i * rowlen + (int64_t)c * NVp + k];
      Y[(int64_t)i * rowlen + (int64_t)c * NVp + k] = a * ft + b * (c == 0 ? M0 : T * M0);
    }
  }
}

// per wall point: wmu[w] = (dJ/drho_w) / N, and the lid-velocity derivative (lid points).
// The interior neighbours and their weights are staged in shared memory; per-thread
// partial sums are in the compute type C (FP32 on the FP32 path: FP64 runs at 1/64 of
// the FP32 rate on this GPU), the block reduction in FP64.
template <typename C, int DIM>
__global__ void __launch_bounds__(256) k_adj_walls(CaseView cv, const C* Y, const C* lam1, double* wmu, double* dtheta) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int NA = 2 + 2 * DIM;
  __shared__ double s_red[RED];
  __shared__ C s_nodes[64];
  __shared__ int32_t s_j[512];
  __shared__ C s_r[512];
  __shared__ int s_mi;
  const int w = blockIdx.x;
  const int b = cv.wall_idx[w];
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int64_t rowlen = (int64_t)NC * NVp;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_nodes[t] = (C)cv.vnodes[t];
  const C* R = reinterpret_cast<const C*>(cv.recon) + (int64_t)b * cap;
  const int32_t* row = cv.col + (int64_t)b * cap;
  if (threadIdx.x < 32) {
    // warp 0 stages the interior neighbours in list order (ballot compaction)
    const int lane = threadIdx.x, m = cv.cnt[b];
    int mi = 0;
    for (int s0 = 0; s0 < m; s0 += 32) {
      const int s = s0 + lane;
      const int j = s < m ? row[s] : 0;
      const bool in = s < m && cv.kind[j] == 0;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = mi + __popc(bal & ((1u << lane) - 1u));
        s_j[pos] = j;
        s_r[pos] = R[s];
      }
      mi += __popc(bal);
    }
    if (lane == 0) s_mi = mi;
  }
  __syncthreads();
  const int mi = s_mi;
  const int8_t* cls = cv.wcls + (int64_t)w * NVp;
  const C* vn = reinterpret_cast<const C*>(cv.wvn) + (int64_t)w * NVp;
  const bool lid = cv.kind[b] == cv.lid_wall;
  const C* Mw = reinterpret_cast<const C*>(cv.mw) + (lid ? NVp : 0);
  const double invN = cv.winv[w];
  const C Tw = (C)cv.wall_T, invTw = (C)(1.0 / cv.wall_T);
  C uw[3] = {(C)0, (C)0, (C)0};
  if (lid)
    for (int a = 0; a < DIM; ++a) uw[a] = (C)cv.lid_u[a];
  C acc[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) acc[q] = (C)0;
  // F = sum over arriving velocities of |v.n| g_b, g_b = sum_j r_bj y_j
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    if (cls[k] != 0) continue;
    C g = (C)0;
    for (int s = 0; s < mi; ++s) g += s_r[s] * Y[(int64_t)s_j[s] * rowlen + k];
    acc[0] += vn[k] * g;
  }
  // mu = sum_{leaving} sum_c lam_c Mw_c ; du_a and dN_a for the lid
  const C* lb = lam1 + (int64_t)b * rowlen;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    if (cls[k] == 0) continue;
    C vd[DIM];
    int kk = k;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { vd[a] = s_nodes[kk % nv]; kk /= nv; }
    const C m0 = Mw[k];
    C lm = lb[k] * m0;
    if (NC == 2) lm += lb[NVp + k] * Tw * m0;
    acc[1] += lm;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const C ca = (vd[a] - uw[a]) * invTw;
      acc[2 + a] += lm * ca;               // sum lam_c Mw_c (v_a - u_a)/T
      acc[2 + DIM + a] += vn[k] * m0 * ca;  // dN/du_a
    }
  }
  double accd[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) accd[q] = (double)acc[q];
  block_reduce<NA>(accd, s_red);
  if (threadIdx.x == 0) {
    const double F = accd[0], mu = accd[1], rho_w = F * invN;
    wmu[w] = mu * invN;
    if (lid)
      for (int a = 0; a < DIM; ++a) atomicAdd(&dtheta[a], rho_w * accd[2 + a] - mu * rho_w * invN * accd[2 + DIM + a]);
  }
}

// per interior point: lam_f~ = VJP of the relaxation applied to lam_y
template <typename C, int DIM>
__global__ void __launch_bounds__(256) k_adj_relax(CaseView cv, const C* FT, const C* lam1, const double* wmu,
                                                   const int32_t* tslot, const int32_t* wall_of, C* LFT, double* dtheta) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  __shared__ double s_red[RED];
  __shared__ double s_nodes[64];
  __shared__ double s_fin[16];
  const int i = cv.int_idx[blockIdx.x];
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp, m = cv.cnt[i];
  const int64_t rowlen = (int64_t)NC * NVp;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_nodes[t] = cv.vnodes[t];
  __syncthreads();
  const C* ft = FT + (int64_t)i * rowlen;
  // moments of f~
  C cpart[DIM + 2];
  for (int q = 0; q < DIM + 2; ++q) cpart[q] = (C)0;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C v2 = (C)0;
    const C g = ft[k];
    cpart[0] += g;
    for (int a = 0; a < DIM; ++a) { cpart[1 + a] += (C)vd[a] * g; v2 += (C)(vd[a] * vd[a]); }
    cpart[DIM + 1] += v2 * g;
    if (NC == 2) cpart[DIM + 1] += ft[NVp + k];
  }
  double part[DIM + 2];
  for (int q = 0; q < DIM + 2; ++q) part[q] = (double)cpart[q];
  block_reduce<DIM + 2>(part, s_red);
  const double pi = 3.14159265358979323846;
  if (threadIdx.x == 0) {
    const double R = part[0];
    double U[3] = {0, 0, 0}, u2 = 0.0;
    for (int a = 0; a < DIM; ++a) { U[a] = part[1 + a] / R; u2 += U[a] * U[a]; }
    const double T = (part[DIM + 1] - R * u2) / (3.0 * R);
    const double wv = cv.wv;
    const double rho = R * wv;
    double tau = 0.0, a = 1.0, b = 0.0, dadtau = 0.0;
    if (cv.tau_mode != 2) {
      tau = cv.tau_mode == 1 ? sqrt(2.0 / pi) * cv.kn : sqrt(2.0 / pi) * cv.kn / (rho * sqrt(T));
      a = tau / (tau + cv.dt);
      b = cv.dt / (tau + cv.dt);
      dadtau = cv.dt / ((tau + cv.dt) * (tau + cv.dt));
    }
    s_fin[0] = R; s_fin[1] = T; s_fin[2] = rho; s_fin[3] = tau; s_fin[4] = a; s_fin[5] = b; s_fin[6] = dadtau;
    s_fin[7] = DIM == 2 ? rho / (2.0 * pi * T) : rho / pow(2.0 * pi * T, 1.5);
    for (int q = 0; q < 3; ++q) s_fin[8 + q] = U[q];
  }
  __syncthreads();
  const C T = (C)s_fin[1], pref = (C)s_fin[7], nl2 = (C)(-0.5 / s_fin[1]);
  C U[DIM];
  for (int d = 0; d < DIM; ++d) U[d] = (C)s_fin[8 + d];
  // lam_y = lam1 + contributions of wall neighbours through their reconstruction; sums for the VJP
  const C* l1 = lam1 + (int64_t)i * rowlen;
  C* lf = LFT + (int64_t)i * rowlen;
  C cs[5 + DIM];  // Af, AM, Sm, Smc2, Sl1, Smc[DIM]
  for (int q = 0; q < 5 + DIM; ++q) cs[q] = (C)0;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    C ly[NC];
    for (int c = 0; c < NC; ++c) ly[c] = l1[(int64_t)c * NVp + k];
    for (int t = 0; t < m; ++t) {
      const int bpt = cv.col[(int64_t)i * cap + t];
      const int w = wall_of[bpt];
      if (w < 0) continue;
      if (cv.wcls[(int64_t)w * NVp + k] != 0) continue;  // leaving velocity of b: not reconstructed
      const int s = tslot[(int64_t)i * cap + t];
      if (s < 0) continue;
      const C r = reinterpret_cast<const C*>(cv.recon)[(int64_t)bpt * cap + s];
      const C* lb = lam1 + (int64_t)bpt * rowlen;
      ly[0] += r * (lb[k] + (C)wmu[w] * reinterpret_cast<const C*>(cv.wvn)[(int64_t)w * NVp + k]);
      if (NC == 2) ly[NC - 1] += r * lb[NVp + k];
    }
    for (int c = 0; c < NC; ++c) lf[(int64_t)c * NVp + k] = ly[c];
    if (cv.tau_mode == 2) continue;
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C c2 = (C)0;
    for (int d = 0; d < DIM; ++d) { const C cc = (C)vd[d] - U[d]; c2 += cc * cc; }
    const C M0 = pref * cexp(nl2 * c2);
    cs[0] += ly[0] * ft[k];
    cs[1] += ly[0] * M0;
    if (NC == 2) {
      cs[0] += ly[NC - 1] * ft[NVp + k];
      cs[1] += ly[NC - 1] * T * M0;
    }
    const C lm = ly[0] + (NC == 2 ? T * ly[NC - 1] : (C)0);
    cs[2] += lm * M0;
    cs[3] += lm * M0 * c2;
    if (NC == 2) cs[4] += ly[NC - 1] * M0;
    for (int d = 0; d < DIM; ++d) cs[5 + d] += lm * M0 * ((C)vd[d] - U[d]);
  }
  if (cv.tau_mode == 2) return;  // lam_f~ = lam_y already written
  double sums[5 + DIM];
  for (int q = 0; q < 5 + DIM; ++q) sums[q] = (double)cs[q];
  block_reduce<5 + DIM>(sums, s_red);
  if (threadIdx.x == 0) {
    const double R = s_fin[0], Td = s_fin[1], rho = s_fin[2], tau = s_fin[3], b = s_fin[5], dadtau = s_fin[6];
    const double Dm = DIM == 2 ? 2.0 : 3.0;
    const double dLda = sums[0] - sums[1];
    double g_rho = b * sums[2] / rho;
    double g_T = b * (sums[3] / (2.0 * Td * Td) - Dm * sums[2] / (2.0 * Td)) + b * sums[4];
    if (cv.tau_mode == 0) {
      g_rho += dLda * dadtau * (-tau / rho);
      g_T += dLda * dadtau * (-tau / (2.0 * Td));
    }
    atomicAdd(&dtheta[3], dLda * dadtau * tau / cv.kn);
    const double wv = cv.wv;
    s_fin[12] = g_rho * wv - g_T * Td / R;  // constant part: g_rho wv - 3 T g_T / (3R)
    s_fin[13] = g_T / (3.0 * R);            // coefficient of |v - U|^2, and the h term
    for (int d = 0; d < DIM; ++d) s_red[d] = b * sums[5 + d] / Td / R;  // g_U_d / R
  }
  __syncthreads();
  const C a = (C)s_fin[4], k0 = (C)s_fin[12], kc2 = (C)s_fin[13];
  C gu[DIM];
  for (int d = 0; d < DIM; ++d) gu[d] = (C)s_red[d];
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C c2 = (C)0, g = k0;
    for (int d = 0; d < DIM; ++d) {
      const C cc = (C)vd[d] - U[d];
      c2 += cc * cc;
      g += gu[d] * cc;
    }
    const C ly0 = lf[k];
    lf[k] = a * ly0 + g + kc2 * c2;
    if (NC == 2) lf[NVp + k] = a * lf[NVp + k] + kc2;
  }
}

// lam0 = L^T lam_f~ (gather over the symmetric neighbour relation)
template <typename C, int DIM>
__global__ void __launch_bounds__(256) k_adj_transport(CaseView cv, const C* LFT, const int32_t* tslot, C* lam0) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  __shared__ double s_nodes[64];
  const int p = blockIdx.x;
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp, m = cv.cnt[p];
  const int64_t rowlen = (int64_t)NC * NVp;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_nodes[t] = cv.vnodes[t];
  __syncthreads();
  const bool interior = cv.kind[p] == 0;
  const C* Pall = reinterpret_cast<const C*>(cv.P);
  const C two_dt = (C)(2.0 * cv.dt);
  for (int k = threadIdx.x; k < NVp; k += blockDim.x) {
    if (k >= NV) {
      for (int c = 0; c < NC; ++c) lam0[(int64_t)p * rowlen + (int64_t)c * NVp + k] = (C)0;
      continue;
    }
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    C v[DIM];
    for (int a = 0; a < DIM; ++a) v[a] = (C)vd[a];
    C diag = (C)0, acc[NC];
    for (int c = 0; c < NC; ++c) acc[c] = (C)0;
    for (int t = 0; t < m; ++t) {
      if (interior) {
        const C* P = Pall + ((int64_t)p * cap + t) * DD;
        C mk = (C)0;
        for (int d = 0; d < DIM; ++d) {
          C pd = (C)0;
          for (int a = 0; a < DIM; ++a) pd += v[a] * P[d * DIM + a];
          mk += cmin(pd, (C)0);
        }
        diag += mk;
      }
      const int i = cv.col[(int64_t)p * cap + t];
      if (cv.kind[i] != 0) continue;
      const int s = tslot[(int64_t)p * cap + t];
      if (s < 0) continue;
      const C* P = Pall + ((int64_t)i * cap + s) * DD;
      C mk = (C)0;
      for (int d = 0; d < DIM; ++d) {
        C pd = (C)0;
        for (int a = 0; a < DIM; ++a) pd += v[a] * P[d * DIM + a];
        mk += cmin(pd, (C)0);
      }
      for (int c = 0; c < NC; ++c) acc[c] += mk * LFT[(int64_t)i * rowlen + (int64_t)c * NVp + k];
    }
    for (int c = 0; c < NC; ++c) {
      const C l = interior ? LFT[(int64_t)p * rowlen + (int64_t)c * NVp + k] : (C)0;
      lam0[(int64_t)p * rowlen + (int64_t)c * NVp + k] = l + two_dt * (diag * l - acc[c]);
    }
  }
}

// objective: J += (1/|lid|) sum_{b in lid} sum_k v_x v_n g_b dv^dim; lam += scale dJ/df
template <typename S, typename C, int DIM>
__global__ void __launch_bounds__(256) k_objective(CaseView cv, int nlid, double* J, C* lam, double scale) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  __shared__ double s_red[RED];
  __shared__ double s_nodes[64];
  const int b = cv.wall_idx[blockIdx.x];
  if (cv.kind[b] != cv.lid_wall) return;  // uniform per block
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) s_nodes[t] = cv.vnodes[t];
  __syncthreads();
  const double wv = cv.wv;
  const S* fb = reinterpret_cast<const S*>(cv.f_in) + (int64_t)b * NC * NVp;
  double acc[1] = {0.0};
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double vd[DIM];
    vel_of<DIM>(k, nv, s_nodes, vd);
    const double wk = vd[0] * vd[DIM - 1] * wv / (double)nlid;
    acc[0] += wk * (double)ld1(fb + k);
    if (lam) lam[(int64_t)b * NC * NVp + k] += (C)(scale * wk);
  }
  block_reduce<1>(acc, s_red);
  if (threadIdx.x == 0 && J) atomicAdd(J, acc[0]);
}

// ---------------------------------------------------------------------------
// FP32 path: warp-per-point adjoint kernels (lanes own 4 velocities of each
// 128-velocity slice, as in the forward transport)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fdiv_small_a(int k, float inv_n) { return (int)(((float)k + 0.5f) * inv_n); }

template <int DIM>
__device__ __forceinline__ void chunk_vel_a(int k0, int nv, int NV, float inv_nv, const float* s_v, float (&vel)[4][DIM],
                                            bool (&kin)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int kk = k0 + e;
    kin[e] = kk < NV;
    if (!kin[e]) kk = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int q = fdiv_small_a(kk, inv_nv);
      vel[e][a] = s_v[kk - q * nv];
      kk = q;
    }
  }
}

__device__ __forceinline__ void ld4f(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void st4f(float* p, const float v[4]) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }

// lam_f~ at interior points from lam1, the wall terms and the relaxation VJP (FP32)
template <int DIM>
__global__ void __launch_bounds__(256) k_adj_relax_wp(CaseView cv, const float* FT, const double* amom, const float* lam1,
                                                      const double* wmu, const int32_t* tslot, const int32_t* wall_of,
                                                      float* LFT, double* dtheta) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  float* s_v = reinterpret_cast<float*>(smem);
  int32_t* s_wb = reinterpret_cast<int32_t*>(smem + 256) + warp * cap * 3;  // (point b, wall slot w, slot of i in b)
  for (int q = threadIdx.x; q < nv; q += blockDim.x) s_v[q] = cv.vnodes_f[q];
  __syncthreads();
  const int t = blockIdx.x * W + warp;
  if (t >= cv.n_int) return;
  const int i = cv.int_idx[t];
  const int m = cv.cnt[i];
  // wall neighbours of i (usually none)
  int nwb = 0;
  for (int q0 = 0; q0 < m; q0 += 32) {
    const int q = q0 + lane;
    int b = -1, w = -1, sl = -1;
    if (q < m) {
      b = cv.col[(int64_t)i * cap + q];
      w = wall_of[b];
      sl = w >= 0 ? tslot[(int64_t)i * cap + q] : -1;
    }
    const bool hit = w >= 0 && sl >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int pos = nwb + __popc(bal & ((1u << lane) - 1u));
      s_wb[3 * pos] = b; s_wb[3 * pos + 1] = w; s_wb[3 * pos + 2] = sl;
    }
    nwb += __popc(bal);
  }
  __syncwarp();
  const double* mo = amom + (int64_t)i * MOM_STRIDE;
  const float rho = (float)mo[0], T = (float)mo[4];
  float U[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) U[a] = (float)mo[1 + a];
  const float wv = cv.wv_f;
  const float R = rho / wv;
  float tau = 0.0f, ca = 1.0f, cb = 0.0f, dadtau = 0.0f;
  if (cv.tau_mode != 2) {
    const float kn = cv.kn_f, dtf = cv.dt_f;
    tau = cv.tau_mode == 1 ? 0.7978845608f * kn : 0.7978845608f * kn / (rho * sqrtf(T));
    ca = tau / (tau + dtf);
    cb = dtf / (tau + dtf);
    dadtau = dtf / ((tau + dtf) * (tau + dtf));
  }
  const float twopiT = 6.283185307f * T;
  const float pref = DIM == 2 ? rho / twopiT : rho / (twopiT * sqrtf(twopiT));
  const float nl2 = -0.5f / T;
  const float inv_nv = 1.0f / (float)nv;
  const int nchunk = NVp >> 2, nslice = (nchunk + 31) >> 5;
  const int64_t rowlen = (int64_t)NC * NVp;
  const float* l1 = lam1 + (int64_t)i * rowlen;
  const float* ft = FT + (int64_t)i * rowlen;
  float* lf = LFT + (int64_t)i * rowlen;
  float cs[5 + DIM];
#pragma unroll
  for (int q = 0; q < 5 + DIM; ++q) cs[q] = 0.0f;
  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = 4 * chunk;
    float vel[4][DIM];
    bool kin[4];
    chunk_vel_a<DIM>(k0, nv, NV, inv_nv, s_v, vel, kin);
    float ly[NC][4], ftv[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) { ld4f(l1 + (int64_t)c * NVp + k0, ly[c]); ld4f(ft + (int64_t)c * NVp + k0, ftv[c]); }
    for (int q = 0; q < nwb; ++q) {
      const int b = s_wb[3 * q], w = s_wb[3 * q + 1], slb = s_wb[3 * q + 2];
      const float r = reinterpret_cast<const float*>(cv.recon)[(int64_t)b * cap + slb];
      const float mu = (float)wmu[w];
      const float* lb = lam1 + (int64_t)b * rowlen + k0;
      const int8_t* cls = cv.wcls + (int64_t)w * NVp + k0;
      const float* vn = reinterpret_cast<const float*>(cv.wvn) + (int64_t)w * NVp + k0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (cls[e] != 0) continue;
        ly[0][e] += r * (lb[e] + mu * vn[e]);
        if (NC == 2) ly[NC - 1][e] += r * lb[NVp + e];
      }
    }
    if (cv.tau_mode == 2) {
#pragma unroll
      for (int c = 0; c < NC; ++c) st4f(lf + (int64_t)c * NVp + k0, ly[c]);
      continue;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!kin[e]) continue;
      float c2 = 0.0f;
      float cc[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) { cc[d] = vel[e][d] - U[d]; c2 = fmaf(cc[d], cc[d], c2); }
      const float M0 = pref * __expf(nl2 * c2);
      cs[0] = fmaf(ly[0][e], ftv[0][e], cs[0]);
      cs[1] = fmaf(ly[0][e], M0, cs[1]);
      float lm = ly[0][e];
      if (NC == 2) {
        cs[0] = fmaf(ly[NC - 1][e], ftv[NC - 1][e], cs[0]);
        cs[1] = fmaf(ly[NC - 1][e], T * M0, cs[1]);
        lm = fmaf(T, ly[NC - 1][e], lm);
        cs[4] = fmaf(ly[NC - 1][e], M0, cs[4]);
      }
      const float lmM = lm * M0;
      cs[2] += lmM;
      cs[3] = fmaf(lmM, c2, cs[3]);
#pragma unroll
      for (int d = 0; d < DIM; ++d) cs[5 + d] = fmaf(lmM, cc[d], cs[5 + d]);
    }
  }
  if (cv.tau_mode == 2) return;
#pragma unroll
  for (int q = 0; q < 5 + DIM; ++q) cs[q] = warp_sum(cs[q]);
  const float Dm = DIM == 2 ? 2.0f : 3.0f;
  const float dLda = cs[0] - cs[1];
  float g_rho = cb * cs[2] / rho;
  float g_T = cb * (cs[3] / (2.0f * T * T) - Dm * cs[2] / (2.0f * T)) + cb * cs[4];
  if (cv.tau_mode == 0) {
    g_rho += dLda * dadtau * (-tau / rho);
    g_T += dLda * dadtau * (-tau / (2.0f * T));
  }
  if (lane == 0) atomicAdd(&dtheta[3], (double)(dLda * dadtau * tau) / cv.kn);
  const float k0c = g_rho * wv - g_T * T / R, kc2 = g_T / (3.0f * R);
  float gu[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) gu[d] = cb * cs[5 + d] / T / R;
  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = 4 * chunk;
    float vel[4][DIM];
    bool kin[4];
    chunk_vel_a<DIM>(k0, nv, NV, inv_nv, s_v, vel, kin);
    float ly[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) ld4f(l1 + (int64_t)c * NVp + k0, ly[c]);
    for (int q = 0; q < nwb; ++q) {  // the wall terms of lam_y again (cheaper than storing lam_y)
      const int b = s_wb[3 * q], w = s_wb[3 * q + 1], slb = s_wb[3 * q + 2];
      const float r = reinterpret_cast<const float*>(cv.recon)[(int64_t)b * cap + slb];
      const float mu = (float)wmu[w];
      const float* lb = lam1 + (int64_t)b * rowlen + k0;
      const int8_t* cls = cv.wcls + (int64_t)w * NVp + k0;
      const float* vn = reinterpret_cast<const float*>(cv.wvn) + (int64_t)w * NVp + k0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (cls[e] != 0) continue;
        ly[0][e] += r * (lb[e] + mu * vn[e]);
        if (NC == 2) ly[NC - 1][e] += r * lb[NVp + e];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float c2 = 0.0f, gsum = k0c;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const float cc = vel[e][d] - U[d];
        c2 = fmaf(cc, cc, c2);
        gsum = fmaf(gu[d], cc, gsum);
      }
      ly[0][e] = kin[e] ? fmaf(ca, ly[0][e], fmaf(kc2, c2, gsum)) : 0.0f;
      if (NC == 2) ly[NC - 1][e] = kin[e] ? fmaf(ca, ly[NC - 1][e], kc2) : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) st4f(lf + (int64_t)c * NVp + k0, ly[c]);
  }
}

// lam0 = L^T lam_f~ (FP32, warp per point, packed FP32x2 as in the forward transport)
template <int DIM>
__global__ void __launch_bounds__(256) k_adj_transport_wp(CaseView cv, const float* LFT, const float* SK, const int32_t* tslot, float* lam0) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  float* s_v = reinterpret_cast<float*>(smem);
  float* s_P = reinterpret_cast<float*>(smem + 256) + (size_t)warp * cap * DD;  // coefficient of p in i's stencil
  int32_t* s_i = reinterpret_cast<int32_t*>(smem + 256 + sizeof(float) * (size_t)W * cap * DD) + warp * cap;
  for (int q = threadIdx.x; q < nv; q += blockDim.x) s_v[q] = cv.vnodes_f[q];
  __syncthreads();
  const int p = blockIdx.x * W + warp;
  if (p >= cv.n) return;
  const int m = cv.cnt[p];
  const bool interior = cv.kind[p] == 0;
  const float* Pall = reinterpret_cast<const float*>(cv.P);
  // stage the transposed coefficients (coefficient of p in the stencil of neighbour i)
  int mt = 0;
  for (int t0 = 0; t0 < m; t0 += 32) {
    const int t = t0 + lane;
    int i = -1, s = -1;
    if (t < m) {
      i = cv.col[(int64_t)p * cap + t];
      s = tslot[(int64_t)p * cap + t];
    }
    const bool use = t < m && s >= 0 && cv.kind[i] == 0;
    const unsigned bal = __ballot_sync(0xffffffffu, use);
    if (use) {
      const int pos = mt + __popc(bal & ((1u << lane) - 1u));
      s_i[pos] = i;
#pragma unroll
      for (int q = 0; q < DD; ++q) s_P[pos * DD + q] = Pall[((int64_t)i * cap + s) * DD + q];
    }
    mt += __popc(bal);
  }
  __syncwarp();
  const float inv_nv = 1.0f / (float)nv;
  const int nchunk = NVp >> 2, nslice = (nchunk + 31) >> 5;
  const int64_t rowlen = (int64_t)NC * NVp;
  const float two_dt = cv.two_dt_f;
  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = 4 * chunk;
    float vel[4][DIM];
    bool kin[4];
    chunk_vel_a<DIM>(k0, nv, NV, inv_nv, s_v, vel, kin);
    float diag[4] = {0.0f, 0.0f, 0.0f, 0.0f}, acc[NC][4];
    if (interior) ld4f(SK + (int64_t)p * NVp + k0, diag);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[c][e] = 0.0f;
    for (int t = 0; t < mt; ++t) {
      const int i = s_i[t];
      float li[NC][4];
#pragma unroll
      for (int c = 0; c < NC; ++c) ld4f(LFT + (int64_t)i * rowlen + (int64_t)c * NVp + k0, li[c]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float mk = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          float pd = vel[e][0] * s_P[t * DD + d * DIM];
#pragma unroll
          for (int a = 1; a < DIM; ++a) pd = fmaf(vel[e][a], s_P[t * DD + d * DIM + a], pd);
          mk += fminf(pd, 0.0f);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c][e] = fmaf(mk, li[c][e], acc[c][e]);
      }
    }
    float own[NC][4], out[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (interior) ld4f(LFT + (int64_t)p * rowlen + (int64_t)c * NVp + k0, own[c]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float l = interior ? own[c][e] : 0.0f;
        out[c][e] = kin[e] ? l + two_dt * (diag[e] * l - acc[c][e]) : 0.0f;
      }
      st4f(lam0 + (int64_t)p * rowlen + (int64_t)c * NVp + k0, out[c]);
    }
  }
}

int launch_adjoint_fp32(const CaseView& cv0, const void* lam1, void* lam0, double* dtheta, void* FT, void* Y, void* LFT,
                        double* wmu, double* amom, float* SK, const int32_t* tslot, const int32_t* wall_of, cudaStream_t s) {
  // forward recomputation with the step's own kernel: y into Y, f~ into FT, the diagonal
  // upwind sums into SK, moments into amom
  CaseView cv = cv0;
  cv.f_out = Y;
  cv.ft_out = (float*)FT;
  cv.sk_out = SK;
  cv.mom = amom;
  int n = launch_transport_fp32(cv, s);
  const int W = 8;
  if (cv.n_wall > 0) {
    if (cv.dim == 2) k_adj_walls<float, 2><<<cv.n_wall, 256, 0, s>>>(cv, (const float*)Y, (const float*)lam1, wmu, dtheta);
    else k_adj_walls<float, 3><<<cv.n_wall, 256, 0, s>>>(cv, (const float*)Y, (const float*)lam1, wmu, dtheta);
    ++n;
  }
  if (cv.n_int > 0) {
    const size_t smem = 256 + sizeof(int32_t) * (size_t)cv.cap * 3 * W;
    const int grid = (cv.n_int + W - 1) / W;
    if (cv.dim == 2) k_adj_relax_wp<2><<<grid, 32 * W, smem, s>>>(cv, (const float*)FT, amom, (const float*)lam1, wmu, tslot, wall_of, (float*)LFT, dtheta);
    else k_adj_relax_wp<3><<<grid, 32 * W, smem, s>>>(cv, (const float*)FT, amom, (const float*)lam1, wmu, tslot, wall_of, (float*)LFT, dtheta);
    ++n;
  }
  {
    const int DD = cv.dim * cv.dim;
    const size_t smem = 256 + sizeof(float) * (size_t)W * cv.cap * DD + sizeof(int32_t) * (size_t)W * cv.cap;
    const int grid = (cv.n + W - 1) / W;
    if (cv.dim == 2) {
      cudaFuncSetAttribute(k_adj_transport_wp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_adj_transport_wp<2><<<grid, 32 * W, smem, s>>>(cv, (const float*)LFT, SK, tslot, (float*)lam0);
    } else {
      cudaFuncSetAttribute(k_adj_transport_wp<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_adj_transport_wp<3><<<grid, 32 * W, smem, s>>>(cv, (const float*)LFT, SK, tslot, (float*)lam0);
    }
    ++n;
  }
  return n;
}

int launch_tslot(const CaseView& cv, int32_t* tslot, cudaStream_t s) {
  k_tslot<<<grid_for(cv.n, 128), 128, 0, s>>>(cv, tslot);
  return 1;
}

template <typename S, typename C, int DIM>
static int adjoint_t(const CaseView& cv, const void* lam1v, void* lam0v, double* dtheta, void* FTv, void* Yv,
                     void* LFTv, double* wmu, const int32_t* tslot, const int32_t* wall_of, cudaStream_t s) {
  C* FT = (C*)FTv;
  C* Y = (C*)Yv;
  C* LFT = (C*)LFTv;
  const C* lam1 = (const C*)lam1v;
  C* lam0 = (C*)lam0v;
  int n = 0;
  if (cv.n_int > 0) { k_adj_prep<S, C, DIM><<<cv.n_int, 256, 0, s>>>(cv, FT, Y); ++n; }
  if (cv.n_wall > 0) { k_adj_walls<C, DIM><<<cv.n_wall, 256, 0, s>>>(cv, Y, lam1, wmu, dtheta); ++n; }
  if (cv.n_int > 0) { k_adj_relax<C, DIM><<<cv.n_int, 256, 0, s>>>(cv, FT, lam1, wmu, tslot, wall_of, LFT, dtheta); ++n; }
  k_adj_transport<C, DIM><<<cv.n, 256, 0, s>>>(cv, LFT, tslot, lam0);
  return n + 1;
}

int launch_adjoint(const CaseView& cv, const void* lam1, void* lam0, double* dtheta, void* FT, void* Y, void* LFT,
                   double* wmu, const int32_t* tslot, const int32_t* wall_of, cudaStream_t s) {
  if (cv.dim == 2) {
    if (cv.storage == 0) return adjoint_t<double, double, 2>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
    if (cv.storage == 1) return adjoint_t<float, float, 2>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
    return adjoint_t<__nv_bfloat16, float, 2>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
  }
  if (cv.storage == 0) return adjoint_t<double, double, 3>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
  if (cv.storage == 1) return adjoint_t<float, float, 3>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
  return adjoint_t<__nv_bfloat16, float, 3>(cv, lam1, lam0, dtheta, FT, Y, LFT, wmu, tslot, wall_of, s);
}

int launch_objective(const CaseView& cv, int nlid, double* J, void* lam, double scale, cudaStream_t s) {
  if (cv.n_wall == 0 || nlid == 0) return 0;
  if (cv.dim == 2) {
    if (cv.storage == 0) k_objective<double, double, 2><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (double*)lam, scale);
    else if (cv.storage == 1) k_objective<float, float, 2><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (float*)lam, scale);
    else k_objective<__nv_bfloat16, float, 2><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (float*)lam, scale);
  } else {
    if (cv.storage == 0) k_objective<double, double, 3><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (double*)lam, scale);
    else if (cv.storage == 1) k_objective<float, float, 3><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (float*)lam, scale);
    else k_objective<__nv_bfloat16, float, 3><<<cv.n_wall, 256, 0, s>>>(cv, nlid, J, (float*)lam, scale);
  }
  return 1;
}

}  // namespace bgk
