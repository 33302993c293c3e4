// Cell-list neighbour search and weighted-least-squares stencils (Sec. 3.4, 3.5.1, 4.2).
//
// Neighbours: counting sort of the points into cells of side >= h, then one
// thread per point scans its own and the adjacent cells and keeps
// j != i with (x_j - x_i).(x_j - x_i) <= h^2, evaluated in FP64 as
// dx*dx + dy*dy (+ dz*dz) left to right without fused multiply-add, so the
// lists are bit-identical to a plain C evaluation.  Rows are kept sorted by
// index (insertion into a thread-private shared-memory row).
//
// Stencils, one thread per point, FP64:
//   interior i:  A = sum_j w_j dr_j dr_j^T, S = A^-1 (closed-form cofactors),
//                coef_j = w_j S dr_j (Eqs. x_derivative..z_derivative),
//                frame n = dr/r; 2D t = (-n_y, n_x); 3D t, b from the spherical
//                angles of dr without trigonometry (phi = atan2(dy, dx),
//                theta = arccos(dz / r); b = (-sin phi, cos phi, 0)),
//                abar_d = e_d . coef_j, stored as P_d = abar_d e_d so that the
//                upwind coefficient is K = sum_d (c.P_d - |c.P_d|).
//   wall b:      linear WLS fit over interior neighbours, p_j = (1, dr_j),
//                recon_j = e_0^T (sum w p p^T)^-1 w_j p_j; with fewer than
//                dim + 1 interior neighbours the constant fit w_j / sum w.
#include <cmath>

#include "bgk_internal.cuh"
#include "device_common.cuh"
#include "nbr_device.cuh"

namespace bgk {

static inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// With sk (ALE skin lists) the cell kernels run only in steps that rebuild the candidates.
__global__ void k_cell_assign(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cv.n) cell_assign_point(cv, i);
}

__global__ void k_cell_scan(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
  cell_scan_block(cv);
}

__global__ void k_cell_fill(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cv.n) cell_fill_point(cv, i);
}

// One warp per point (see nbr_warp_point).
template <int DIM, bool CAND>
__global__ void __launch_bounds__(256) k_neighbours_warp(CaseView cv, float lo, float hi) {
  extern __shared__ int32_t s_buf[];  // [W][cap]
  if (CAND && !cv.sk->rebuild) return;
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * W + warp;
  if (i >= cv.n) return;  // whole warp leaves together
  nbr_warp_point<DIM, CAND>(cv, i, lane, s_buf + warp * (CAND ? cv.ccap : cv.cap), lo, hi);
}

// One warp per point (see filter_warp_point).
template <int DIM>
__global__ void __launch_bounds__(256) k_filter(CaseView cv, float lo, float hi) {
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * W + warp;
  // the candidate build of this list build (if any) has consumed the rebuild flag
  if (blockIdx.x == 0 && threadIdx.x == 0 && cv.sk) cv.sk->rebuild = 0;
  if (i >= cv.n) return;
  filter_warp_point<DIM>(cv, i, lane, lo, hi);
}

// FP32 prefilter bounds for radius r: squared distances below lo are inside, above
// hi outside, in between the FP64 test decides.
static void prefilter_bounds(int dim, double r, float* lo, float* hi) {
  const double r2 = r * r;
  const double band = 8.0 * dim * std::ldexp(1.0, -22) / r + std::ldexp(1.0, -16);
  *lo = band < 1.0 ? (float)(r2 * (1.0 - band)) : -1.0f;
  *hi = (float)(r2 * (1.0 + band));
}

int launch_neighbours(const CaseView& cv, cudaStream_t s) {
  cudaMemsetAsync(cv.cell_cnt, 0, sizeof(int32_t) * cv.ncell, s);
  k_cell_assign<<<grid_for(cv.n, 256), 256, 0, s>>>(cv, nullptr);
  k_cell_scan<<<1, 1024, 0, s>>>(cv, nullptr);
  k_cell_fill<<<grid_for(cv.n, 256), 256, 0, s>>>(cv, nullptr);
  const int W = 8;
  const size_t smem = sizeof(int32_t) * (size_t)cv.cap * W;
  float lo, hi;
  prefilter_bounds(cv.dim, cv.h, &lo, &hi);
  if (cv.dim == 2) k_neighbours_warp<2, false><<<grid_for(cv.n, W), 32 * W, smem, s>>>(cv, lo, hi);
  else k_neighbours_warp<3, false><<<grid_for(cv.n, W), 32 * W, smem, s>>>(cv, lo, hi);
  return 4;
}

int launch_neighbours_skin(const CaseView& cv, cudaStream_t s) {
  k_cell_assign<<<grid_for(cv.n, 256), 256, 0, s>>>(cv, cv.sk);
  k_cell_scan<<<1, 1024, 0, s>>>(cv, cv.sk);
  k_cell_fill<<<grid_for(cv.n, 256), 256, 0, s>>>(cv, cv.sk);
  const int W = 8;
  const size_t smem = sizeof(int32_t) * (size_t)cv.ccap * W;
  float clo, chi, lo, hi;
  prefilter_bounds(cv.dim, cv.h * (1.0 + cv.skin), &clo, &chi);
  prefilter_bounds(cv.dim, cv.h, &lo, &hi);
  if (cv.dim == 2) {
    auto kc = k_neighbours_warp<2, true>;
    cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kc<<<grid_for(cv.n, W), 32 * W, smem, s>>>(cv, clo, chi);
    k_filter<2><<<grid_for(cv.n, W), 32 * W, 0, s>>>(cv, lo, hi);
  } else {
    auto kc = k_neighbours_warp<3, true>;
    cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kc<<<grid_for(cv.n, W), 32 * W, smem, s>>>(cv, clo, chi);
    k_filter<3><<<grid_for(cv.n, W), 32 * W, 0, s>>>(cv, lo, hi);
  }
  return 6;
}

// ---- stencils ----

// Solve the symmetric m x m system B z = e_0 by Gaussian elimination with partial
// pivoting; returns false when a pivot is not above 1e-12 * max|B|.
template <int M>
__device__ bool solve_e0(double (&B)[M][M], double (&z)[M]) {
  double rhs[M];
  double amax = 0.0;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    rhs[r] = r == 0 ? 1.0 : 0.0;
#pragma unroll
    for (int c = 0; c < M; ++c) amax = fmax(amax, fabs(B[r][c]));
  }
  if (!(amax > 0.0)) return false;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    int piv = c;
#pragma unroll
    for (int r = c + 1; r < M; ++r)
      if (fabs(B[r][c]) > fabs(B[piv][c])) piv = r;
    if (!(fabs(B[piv][c]) > 1e-12 * amax)) return false;
    if (piv != c) {
#pragma unroll
      for (int k = 0; k < M; ++k) { double tmp = B[c][k]; B[c][k] = B[piv][k]; B[piv][k] = tmp; }
      double tmp = rhs[c]; rhs[c] = rhs[piv]; rhs[piv] = tmp;
    }
#pragma unroll
    for (int r = c + 1; r < M; ++r) {
      double fct = B[r][c] / B[c][c];
#pragma unroll
      for (int k = c; k < M; ++k) B[r][k] -= fct * B[c][k];
      rhs[r] -= fct * rhs[c];
    }
  }
#pragma unroll
  for (int r = M - 1; r >= 0; --r) {
    double acc = rhs[r];
#pragma unroll
    for (int k = r + 1; k < M; ++k) acc -= B[r][k] * z[k];
    z[r] = acc / B[r][r];
  }
  return true;
}

// Interior stencil of the second-order Taylor fit (Sec. 3.4.1, higher-order
// approximation), FP64, one thread per point: basis b_j = (dr, dr_a dr_b for a <= b,
// halved on the diagonal), B = sum_j w_j b_j b_j^T (MQ x MQ, MQ = dim + dim (dim + 1) / 2),
// G = the first dim columns of B^-1 by Gauss-Jordan elimination with partial pivoting
// on [B | e_0 .. e_{dim-1}] (B is symmetric, so they are its gradient rows), coef_j =
// w_j G^T b_j; frames and projected coefficients as for the linear fit.
template <int DIM>
__device__ __forceinline__ void quad_basis_d(const double* xi, const double* xj, int periodic, double* b, double* dr) {
  for (int a = 0; a < DIM; ++a) dr[a] = sep_d(xi[a], xj[a], periodic);
  int k = 0;
  for (int a = 0; a < DIM; ++a) b[k++] = dr[a];
  for (int a = 0; a < DIM; ++a)
    for (int c = a; c < DIM; ++c) b[k++] = a == c ? 0.5 * dr[a] * dr[a] : dr[a] * dr[c];
}

template <typename C, int DIM>
__device__ void quad_stencil_point(const CaseView& cv, const int i, const double* xi, const int32_t* row,
                                   const int m, C* P) {
  constexpr int MQ = DIM + DIM * (DIM + 1) / 2;
  const double nah2 = -cv.alpha, hh = cv.h * cv.h;
  double B[MQ][MQ + DIM];
  for (int a = 0; a < MQ; ++a)
    for (int c = 0; c < MQ + DIM; ++c) B[a][c] = 0.0;
  for (int s = 0; s < m; ++s) {
    double xj[DIM], b[MQ], dr[DIM];
    for (int a = 0; a < DIM; ++a) xj[a] = cv.x[(int64_t)row[s] * DIM + a];
    quad_basis_d<DIM>(xi, xj, cv.periodic, b, dr);
    const double w = exp(nah2 * dist2_d<DIM>(xi, xj, cv.periodic) / hh);
    for (int a = 0; a < MQ; ++a)
      for (int c = 0; c < MQ; ++c) B[a][c] += w * b[a] * b[c];
  }
  double amax = 0.0;
  for (int a = 0; a < MQ; ++a) {
    for (int c = 0; c < MQ; ++c) amax = fmax(amax, fabs(B[a][c]));
    for (int c = 0; c < DIM; ++c) B[a][MQ + c] = a == c ? 1.0 : 0.0;
  }
  bool ok = m >= MQ && amax > 0.0;
  for (int c = 0; c < MQ && ok; ++c) {
    int piv = c;
    for (int r = c + 1; r < MQ; ++r)
      if (fabs(B[r][c]) > fabs(B[piv][c])) piv = r;
    if (!(fabs(B[piv][c]) > 1e-12 * amax)) { ok = false; break; }
    if (piv != c)
      for (int k = 0; k < MQ + DIM; ++k) { const double t = B[c][k]; B[c][k] = B[piv][k]; B[piv][k] = t; }
    const double d = B[c][c];
    for (int k = 0; k < MQ + DIM; ++k) B[c][k] /= d;
    for (int r = 0; r < MQ; ++r) {
      if (r == c) continue;
      const double f = B[r][c];
      for (int k = 0; k < MQ + DIM; ++k) B[r][k] -= f * B[c][k];
    }
  }
  if (!ok) {
    set_status(cv.status, ST_SINGULAR);
    for (int s = 0; s < m * DIM * DIM; ++s) P[s] = (C)0;
    return;
  }
  for (int s = 0; s < m; ++s) {
    double xj[DIM], b[MQ], dr[DIM];
    for (int a = 0; a < DIM; ++a) xj[a] = cv.x[(int64_t)row[s] * DIM + a];
    quad_basis_d<DIM>(xi, xj, cv.periodic, b, dr);
    const double r2 = dist2_d<DIM>(xi, xj, cv.periodic);
    const double w = exp(nah2 * r2 / hh);
    double coef[DIM];
    for (int a = 0; a < DIM; ++a) {
      double acc = 0.0;
      for (int c = 0; c < MQ; ++c) acc += B[c][MQ + a] * b[c];
      coef[a] = w * acc;
    }
    const double r = sqrt(r2);
    double E[DIM][DIM];  // rows n, t(, b)
    if constexpr (DIM == 2) {
      const double nx = dr[0] / r, ny = dr[1] / r;
      E[0][0] = nx; E[0][1] = ny;
      E[1][0] = -ny; E[1][1] = nx;
    } else {
      const double rxy = sqrt(dr[0] * dr[0] + dr[1] * dr[1]);
      const double cphi = rxy > 0.0 ? dr[0] / rxy : 1.0, sphi = rxy > 0.0 ? dr[1] / rxy : 0.0;
      const double cth = dr[2] / r, sth = rxy / r;
      E[0][0] = dr[0] / r; E[0][1] = dr[1] / r; E[0][2] = dr[2] / r;
      E[1][0] = cth * cphi; E[1][1] = cth * sphi; E[1][2] = -sth;
      E[2][0] = -sphi; E[2][1] = cphi; E[2][2] = 0.0;
    }
    for (int d = 0; d < DIM; ++d) {
      double ab = 0.0;
      for (int a = 0; a < DIM; ++a) ab += E[d][a] * coef[a];
      for (int a = 0; a < DIM; ++a) P[(s * DIM + d) * DIM + a] = (C)(ab * E[d][a]);
    }
  }
}

template <typename C, int DIM>
__global__ void k_stencils(CaseView cv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int cap = cv.cap, m = cv.cnt[i];
  const int32_t* row = cv.col + (int64_t)i * cap;
  double xi[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xi[a] = cv.x[(int64_t)i * DIM + a];
  const double nah2 = -cv.alpha, hh = cv.h * cv.h;
  C* P = (C*)cv.P + (int64_t)i * cap * DIM * DIM;
  C* R = (C*)cv.recon + (int64_t)i * cap;
  if (cv.kind[i] == 0 && cv.wls_order == 2) {
    quad_stencil_point<C, DIM>(cv, i, xi, row, m, P);
  } else if (cv.kind[i] == 0) {
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      double dr[DIM], xj[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; dr[a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double w = exp(nah2 * dist2_d<DIM>(xi, xj, cv.periodic) / hh);
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) A[a][b] += w * dr[a] * dr[b];
    }
    double S[3][3];
    double det, scale = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) scale = fmax(scale, fabs(A[a][a]));
    if constexpr (DIM == 2) {
      det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      S[0][0] = A[1][1] / det; S[0][1] = -A[0][1] / det;
      S[1][0] = -A[1][0] / det; S[1][1] = A[0][0] / det;
    } else {
      const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
      const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
      const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
      det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
      S[0][0] = c00 / det;
      S[1][0] = c01 / det;
      S[2][0] = c02 / det;
      S[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
      S[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
      S[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
      S[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
      S[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
      S[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    }
    double sc = 1.0;
    for (int a = 0; a < DIM; ++a) sc *= scale;
    if (m < DIM || !(fabs(det) > 1e-12 * sc) || !isfinite(det)) {
      set_status(cv.status, ST_SINGULAR);
      for (int s = 0; s < m * DIM * DIM; ++s) P[s] = (C)0;
      return;
    }
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      double dr[DIM], xj[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; dr[a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double r2 = dist2_d<DIM>(xi, xj, cv.periodic);
      const double w = exp(nah2 * r2 / hh);
      double coef[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) acc += S[a][b] * dr[b];
        coef[a] = w * acc;
      }
      const double r = sqrt(r2);
      double E[DIM][DIM];  // rows n, t(, b)
      if constexpr (DIM == 2) {
        const double nx = dr[0] / r, ny = dr[1] / r;
        E[0][0] = nx; E[0][1] = ny;
        E[1][0] = -ny; E[1][1] = nx;
      } else {
        const double rxy = sqrt(dr[0] * dr[0] + dr[1] * dr[1]);
        const double cphi = rxy > 0.0 ? dr[0] / rxy : 1.0, sphi = rxy > 0.0 ? dr[1] / rxy : 0.0;
        const double cth = dr[2] / r, sth = rxy / r;
        E[0][0] = dr[0] / r; E[0][1] = dr[1] / r; E[0][2] = dr[2] / r;
        E[1][0] = cth * cphi; E[1][1] = cth * sphi; E[1][2] = -sth;
        E[2][0] = -sphi; E[2][1] = cphi; E[2][2] = 0.0;
      }
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double ab = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) ab += E[d][a] * coef[a];
#pragma unroll
        for (int a = 0; a < DIM; ++a) P[(s * DIM + d) * DIM + a] = (C)(ab * E[d][a]);
      }
    }
  } else {
    constexpr int M = DIM + 1;
    double B[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int b = 0; b < M; ++b) B[a][b] = 0.0;
    int ninner = 0;
    double wsum = 0.0;
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      if (cv.kind[j] != 0) continue;
      double pj[M], xj[DIM];
      pj[0] = 1.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; pj[1 + a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double w = exp(nah2 * dist2_d<DIM>(xi, xj, cv.periodic) / hh);
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) B[a][b] += w * pj[a] * pj[b];
      wsum += w;
      ++ninner;
    }
    double z[M];
    const bool linear = ninner >= M;
    if (ninner == 0 || (linear && !solve_e0<M>(B, z))) {
      set_status(cv.status, ST_SINGULAR);
      for (int s = 0; s < m; ++s) R[s] = (C)0;
      return;
    }
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      if (cv.kind[j] != 0) { R[s] = (C)0; continue; }
      double pj[M], xj[DIM];
      pj[0] = 1.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; pj[1 + a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double w = exp(nah2 * dist2_d<DIM>(xi, xj, cv.periodic) / hh);
      double r;
      if (linear) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < M; ++b) acc += z[b] * pj[b];
        r = w * acc;
      } else {
        r = w / wsum;
      }
      R[s] = (C)r;
    }
  }
}

// Interior stencils of the FP32/BF16 path, LPP lanes per point (stencil_grp_point),
// points in the interior list order.
template <int DIM, int LPP>
__global__ void __launch_bounds__(256) k_stencils_grp(CaseView cv) {
  const int gid = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPP);
  const bool valid = gid < cv.n_int;
  stencil_grp_point<DIM, LPP>(cv, valid ? cv.int_idx[gid] : 0, valid, threadIdx.x % LPP);
}

// FP32/BF16 path, wall points: linear WLS reconstruction weights, a group of
// LPP lanes per wall point; B = sum w p p^T with p = (1, dr/h) accumulated in
// FP32 and reduced by shuffles, the (dim+1)^2 system solved in FP64 by the
// group's first lane (scaling the linear part of the basis leaves the weights
// unchanged and keeps the entries of B of order one).
template <int DIM, int LPP>
__global__ void __launch_bounds__(256) k_recon_grp(CaseView cv) {
  constexpr int M = DIM + 1;
  constexpr int NB = M * (M + 1) / 2;
  const int gid = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPP);
  const int sub = threadIdx.x % LPP;
  const bool valid = gid < cv.n_wall;
  const int i = valid ? cv.wall_idx[gid] : 0;
  const int m = valid ? cv.cnt[i] : 0;
  const int cap = cv.cap;
  const int32_t* row = cv.col + (int64_t)i * cap;
  const float nah2 = cv.nah2_f;
  const float inv_h = cv.inv_h_f;  // basis (1, dr/h): same weights, O(1) matrix entries
  float B[NB], wsum = 0.0f;
  int ninner = 0;
#pragma unroll
  for (int q = 0; q < NB; ++q) B[q] = 0.0f;
  for (int s = sub; s < m; s += LPP) {
    const int j = row[s];
    if (cv.kind[j] != 0) continue;
    float p[M], r2 = 0.0f;
    float dr[DIM];
    sep_hilo<DIM>(cv, i, j, dr);
    p[0] = 1.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { p[1 + a] = dr[a] * inv_h; r2 = fmaf(dr[a], dr[a], r2); }
    const float w = expf(nah2 * r2);
    int q = 0;
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int b = a; b < M; ++b) { B[q] = fmaf(w * p[a], p[b], B[q]); ++q; }
    wsum += w;
    ++ninner;
  }
#pragma unroll
  for (int o = LPP / 2; o >= 1; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NB; ++q) B[q] += __shfl_xor_sync(0xffffffffu, B[q], o);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    ninner += __shfl_xor_sync(0xffffffffu, ninner, o);
  }
  float zf[M];
  int ok = 1;
  if (sub == 0) {
    double Bd[M][M], z[M];
    int q = 0;
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int b = a; b < M; ++b) { Bd[a][b] = (double)B[q]; Bd[b][a] = (double)B[q]; ++q; }
    ok = valid && ninner > 0;
    if (ok && ninner >= M) ok = solve_e0<M>(Bd, z);
#pragma unroll
    for (int a = 0; a < M; ++a) zf[a] = ok && ninner >= M ? (float)z[a] : 0.0f;
  }
  const int src = (threadIdx.x & 31) & ~(LPP - 1);
#pragma unroll
  for (int a = 0; a < M; ++a) zf[a] = __shfl_sync(0xffffffffu, zf[a], src);
  ok = __shfl_sync(0xffffffffu, ok, src);
  if (!valid) return;
  float* R = (float*)cv.recon + (int64_t)i * cap;
  if (!ok) {
    if (sub == 0) set_status(cv.status, ST_SINGULAR);
    for (int s = sub; s < m; s += LPP) R[s] = 0.0f;
    return;
  }
  const bool linear = ninner >= M;
  for (int s = sub; s < m; s += LPP) {
    const int j = row[s];
    if (cv.kind[j] != 0) { R[s] = 0.0f; continue; }
    float dr[DIM];
    sep_hilo<DIM>(cv, i, j, dr);
    float r2 = 0.0f, acc = zf[0];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { r2 = fmaf(dr[a], dr[a], r2); acc = fmaf(zf[1 + a], dr[a] * inv_h, acc); }
    const float w = expf(nah2 * r2);
    R[s] = linear ? w * acc : w / wsum;
  }
}

int launch_stencils(const CaseView& cv, cudaStream_t s, int part) {
  const int B = 128;
  const bool f64 = cv.storage == 0;
  if (f64 || cv.wls_order == 2) {
    // one FP64 thread per point for every point (the second-order fit: also for
    // FP32/BF16 storage, the coefficients then rounded to FP32)
    if (part == 2) return 0;
    if (f64) {
      if (cv.dim == 2) k_stencils<double, 2><<<grid_for(cv.n, B), B, 0, s>>>(cv);
      else k_stencils<double, 3><<<grid_for(cv.n, B), B, 0, s>>>(cv);
    } else {
      if (cv.dim == 2) k_stencils<float, 2><<<grid_for(cv.n, B), B, 0, s>>>(cv);
      else k_stencils<float, 3><<<grid_for(cv.n, B), B, 0, s>>>(cv);
    }
    return 1;
  }
  constexpr int LPP = 4;
  int n = 0;
  if (cv.n_int > 0 && part != 2) {
    const int grid = grid_for((int64_t)cv.n_int * LPP, 256);
    if (cv.dim == 2) k_stencils_grp<2, LPP><<<grid, 256, 0, s>>>(cv);
    else k_stencils_grp<3, LPP><<<grid, 256, 0, s>>>(cv);
    ++n;
  }
  if (cv.n_wall > 0 && part != 1) {
    const int grid = grid_for((int64_t)cv.n_wall * LPP, 128);
    if (cv.dim == 2) k_recon_grp<2, LPP><<<grid, 128, 0, s>>>(cv);
    else k_recon_grp<3, LPP><<<grid, 128, 0, s>>>(cv);
    ++n;
  }
  return n;
}

// Copy the stencils of every neighbour slot into CSR-ordered double arrays
// (rowptr computed on the host from cnt).
template <typename C>
__global__ void k_stencils_to_double(CaseView cv, const int64_t* rowptr, double* Pout, double* Rout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int DD = cv.dim * cv.dim, m = cv.cnt[i];
  const C* P = (const C*)cv.P + (int64_t)i * cv.cap * DD;
  const C* R = (const C*)cv.recon + (int64_t)i * cv.cap;
  const int64_t o = rowptr[i];
  const bool interior = cv.kind[i] == 0;
  for (int s = 0; s < m; ++s) {
    for (int q = 0; q < DD; ++q) Pout[(o + s) * DD + q] = interior ? (double)P[s * DD + q] : 0.0;
    Rout[o + s] = interior ? 0.0 : (double)R[s];
  }
}

int launch_stencils_csr(const CaseView& cv, const int64_t* rowptr, double* P, double* recon, cudaStream_t s) {
  const int B = 128;
  if (cv.storage == 0) k_stencils_to_double<double><<<grid_for(cv.n, B), B, 0, s>>>(cv, rowptr, P, recon);
  else k_stencils_to_double<float><<<grid_for(cv.n, B), B, 0, s>>>(cv, rowptr, P, recon);
  return 1;
}

}  // namespace bgk
