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

namespace bgk {

static inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

__global__ void k_cell_assign(CaseView cv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  int c = 0, stride = 1;
  for (int a = 0; a < cv.dim; ++a) {
    int ca = (int)floor(__dmul_rn(cv.x[(int64_t)i * cv.dim + a], (double)cv.nc));
    ca = ca < 0 ? 0 : (ca > cv.nc - 1 ? cv.nc - 1 : ca);
    c += ca * stride;
    stride *= cv.nc;
  }
  cv.cell_of[i] = c;
  atomicAdd(&cv.cell_cnt[c], 1);
  for (int a = 0; a < cv.dim; ++a) cv.xf[(int64_t)i * cv.dim + a] = (float)cv.x[(int64_t)i * cv.dim + a];
}

// Exclusive scan of the cell counts into cell_start (one block), then clear the counts.
__global__ void k_cell_scan(CaseView cv) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int ncell = cv.ncell;
  const int per = (ncell + T - 1) / T;
  const int lo = t * per, hi = min(lo + per, ncell);
  int32_t s = 0;
  for (int c = lo; c < hi; ++c) s += cv.cell_cnt[c];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;  // exclusive prefix of this thread's range
  for (int c = lo; c < hi; ++c) {
    cv.cell_start[c] = run;
    run += cv.cell_cnt[c];
    cv.cell_cnt[c] = 0;
  }
  if (t == T - 1) cv.cell_start[ncell] = part[T - 1];
}

__global__ void k_cell_fill(CaseView cv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  int c = cv.cell_of[i];
  int pos = cv.cell_start[c] + atomicAdd(&cv.cell_cnt[c], 1);
  cv.cell_pts[pos] = i;
}

// Candidate test: the FP32 squared distance decides unless it lies within a
// relative band of h^2 that bounds its rounding error (positions rounded to
// FP32: |dx_f - dx| <= 2^-23 + 2^-24 |dx|, so |d2_f - d2| <= dim 2^-22 h + O(2^-23 h^2)
// near the cut; the band is 8x that); candidates inside the band take the exact
// FP64 test.  The result equals the FP64 test for every pair.
template <int DIM>
__global__ void k_neighbours(CaseView cv, float lo, float hi) {
  extern __shared__ int32_t s_row[];  // [cap][blockDim] strided thread-private rows
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int B = blockDim.x, t = threadIdx.x, cap = cv.cap, nc = cv.nc;
  float xif[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xif[a] = cv.xf[(int64_t)i * DIM + a];
  const double h2 = __dmul_rn(cv.h, cv.h);
  int ci[3] = {0, 0, 0};
  {
    int r = cv.cell_of[i];
    for (int a = 0; a < DIM; ++a) { ci[a] = r % nc; r /= nc; }
  }
  int lst[3][3], len[3];
  for (int a = 0; a < 3; ++a) { len[a] = 1; lst[a][0] = 0; lst[a][1] = 0; lst[a][2] = 0; }
  for (int a = 0; a < DIM; ++a) {
    len[a] = 0;
    if (cv.periodic && nc < 3) {
      for (int c = 0; c < nc; ++c) lst[a][len[a]++] = c;
    } else {
      for (int o = -1; o <= 1; ++o) {
        int c = ci[a] + o;
        if (cv.periodic) c = (c + nc) % nc;
        else if (c < 0 || c >= nc) continue;
        lst[a][len[a]++] = c;
      }
    }
  }
  int m = 0;
  for (int u = 0; u < len[2]; ++u)
    for (int v = 0; v < len[1]; ++v)
      for (int w = 0; w < len[0]; ++w) {
        int c = lst[0][w];
        if (DIM >= 2) c += lst[1][v] * nc;
        if (DIM >= 3) c += lst[2][u] * nc * nc;
        const int q0 = cv.cell_start[c], q1 = cv.cell_start[c + 1];
        for (int q = q0; q < q1; ++q) {
          const int j = cv.cell_pts[q];
          if (j == i) continue;
          float d2f = 0.0f;
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            float d = cv.xf[(int64_t)j * DIM + a] - xif[a];
            if (cv.periodic) d = d > 0.5f ? d - 1.0f : (d < -0.5f ? d + 1.0f : d);
            d2f = fmaf(d, d, d2f);
          }
          if (d2f > hi) continue;
          bool inside = d2f <= lo;
          if (!inside) {
            double xi[DIM], xj[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) { xi[a] = cv.x[(int64_t)i * DIM + a]; xj[a] = cv.x[(int64_t)j * DIM + a]; }
            inside = dist2_d<DIM>(xi, xj, cv.periodic) <= h2;
          }
          if (inside) {
            if (m < cap) {
              int p = m;
              while (p > 0 && s_row[(p - 1) * B + t] > j) {
                s_row[p * B + t] = s_row[(p - 1) * B + t];
                --p;
              }
              s_row[p * B + t] = j;
            }
            ++m;
          }
        }
      }
  const int mm = m < cap ? m : cap;
  int32_t* row = cv.col + (int64_t)i * cap;
  for (int p = 0; p < mm; ++p) row[p] = s_row[p * B + t];
  cv.cnt[i] = mm;
  if (m > cap) set_status(cv.status, ST_OVERFLOW);
  atomicAdd(&cv.status->nnz, (unsigned long long)m);
}

int launch_neighbours(const CaseView& cv, cudaStream_t s) {
  const int B = 128;
  cudaMemsetAsync(cv.cell_cnt, 0, sizeof(int32_t) * cv.ncell, s);
  k_cell_assign<<<grid_for(cv.n, 256), 256, 0, s>>>(cv);
  k_cell_scan<<<1, 1024, 0, s>>>(cv);
  k_cell_fill<<<grid_for(cv.n, 256), 256, 0, s>>>(cv);
  size_t smem = sizeof(int32_t) * (size_t)cv.cap * B;
  const double h2 = cv.h * cv.h;
  const double band = 8.0 * cv.dim * std::ldexp(1.0, -22) / cv.h + std::ldexp(1.0, -16);
  const float lo = band < 1.0 ? (float)(h2 * (1.0 - band)) : -1.0f;
  const float hi = (float)(h2 * (1.0 + band));
  if (cv.dim == 2) {
    cudaFuncSetAttribute(k_neighbours<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_neighbours<2><<<grid_for(cv.n, B), B, smem, s>>>(cv, lo, hi);
  } else {
    cudaFuncSetAttribute(k_neighbours<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_neighbours<3><<<grid_for(cv.n, B), B, smem, s>>>(cv, lo, hi);
  }
  return 4;
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
  if (cv.kind[i] == 0) {
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

// FP32/BF16 path: the normal matrix A = sum w dr dr^T and its inverse stay in
// FP64; the weights, gradient coefficients and frames are evaluated in FP32
// (they are stored in FP32), which keeps FP64 work to a few operations per pair.
template <int DIM>
__global__ void k_stencils_f32(CaseView cv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int cap = cv.cap, m = cv.cnt[i];
  const int32_t* row = cv.col + (int64_t)i * cap;
  double xi[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xi[a] = cv.x[(int64_t)i * DIM + a];
  const float nah2 = (float)(-cv.alpha / (cv.h * cv.h));
  float* P = (float*)cv.P + (int64_t)i * cap * DIM * DIM;
  float* R = (float*)cv.recon + (int64_t)i * cap;
  if (cv.kind[i] == 0) {
    double A[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) A[a][b] = 0.0;
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      float dr[DIM];
      float r2 = 0.0f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        dr[a] = (float)sep_d(xi[a], cv.x[(int64_t)j * DIM + a], cv.periodic);
        r2 += dr[a] * dr[a];
      }
      const float w = expf(nah2 * r2);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float wa = w * dr[a];
#pragma unroll
        for (int b = a; b < DIM; ++b) A[a][b] += (double)wa * (double)dr[b];
      }
    }
    float S[DIM][DIM];
    double det, scale = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) scale = fmax(scale, fabs(A[a][a]));
    if constexpr (DIM == 2) {
      det = A[0][0] * A[1][1] - A[0][1] * A[0][1];
      const double id = 1.0 / det;
      S[0][0] = (float)(A[1][1] * id); S[0][1] = (float)(-A[0][1] * id);
      S[1][0] = S[0][1]; S[1][1] = (float)(A[0][0] * id);
    } else {
      const double c00 = A[1][1] * A[2][2] - A[1][2] * A[1][2];
      const double c01 = A[1][2] * A[0][2] - A[0][1] * A[2][2];
      const double c02 = A[0][1] * A[1][2] - A[1][1] * A[0][2];
      det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
      const double id = 1.0 / det;
      S[0][0] = (float)(c00 * id); S[0][1] = (float)(c01 * id); S[0][2] = (float)(c02 * id);
      S[1][1] = (float)((A[0][0] * A[2][2] - A[0][2] * A[0][2]) * id);
      S[1][2] = (float)((A[0][1] * A[0][2] - A[0][0] * A[1][2]) * id);
      S[2][2] = (float)((A[0][0] * A[1][1] - A[0][1] * A[0][1]) * id);
      S[1][0] = S[0][1]; S[2][0] = S[0][2]; S[2][1] = S[1][2];
    }
    if (m < DIM || !(fabs(det) > 1e-12 * pow(scale, (double)DIM)) || !isfinite(det)) {
      set_status(cv.status, ST_SINGULAR);
      for (int s = 0; s < m * DIM * DIM; ++s) P[s] = 0.0f;
      return;
    }
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      float dr[DIM];
      float r2 = 0.0f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        dr[a] = (float)sep_d(xi[a], cv.x[(int64_t)j * DIM + a], cv.periodic);
        r2 += dr[a] * dr[a];
      }
      const float w = expf(nah2 * r2);
      float coef[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float acc = 0.0f;
#pragma unroll
        for (int b = 0; b < DIM; ++b) acc += S[a][b] * dr[b];
        coef[a] = w * acc;
      }
      const float rinv = 1.0f / sqrtf(r2);
      float E[DIM][DIM];
      if constexpr (DIM == 2) {
        const float nx = dr[0] * rinv, ny = dr[1] * rinv;
        E[0][0] = nx; E[0][1] = ny;
        E[1][0] = -ny; E[1][1] = nx;
      } else {
        const float rxy = sqrtf(dr[0] * dr[0] + dr[1] * dr[1]);
        const float cphi = rxy > 0.0f ? dr[0] / rxy : 1.0f, sphi = rxy > 0.0f ? dr[1] / rxy : 0.0f;
        const float cth = dr[2] * rinv, sth = rxy * rinv;
        E[0][0] = dr[0] * rinv; E[0][1] = dr[1] * rinv; E[0][2] = cth;
        E[1][0] = cth * cphi; E[1][1] = cth * sphi; E[1][2] = -sth;
        E[2][0] = -sphi; E[2][1] = cphi; E[2][2] = 0.0f;
      }
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        float ab = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) ab += E[d][a] * coef[a];
#pragma unroll
        for (int a = 0; a < DIM; ++a) P[(s * DIM + d) * DIM + a] = ab * E[d][a];
      }
    }
  } else {
    // wall reconstruction: small (dim+1)^2 solve per wall point, kept in FP64
    constexpr int M = DIM + 1;
    double B[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int b = 0; b < M; ++b) B[a][b] = 0.0;
    int ninner = 0;
    double wsum = 0.0;
    const double nah2d = -cv.alpha / (cv.h * cv.h);
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      if (cv.kind[j] != 0) continue;
      double pj[M], xj[DIM];
      pj[0] = 1.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; pj[1 + a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double w = exp(nah2d * dist2_d<DIM>(xi, xj, cv.periodic));
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
      for (int s = 0; s < m; ++s) R[s] = 0.0f;
      return;
    }
    for (int s = 0; s < m; ++s) {
      const int j = row[s];
      if (cv.kind[j] != 0) { R[s] = 0.0f; continue; }
      double pj[M], xj[DIM];
      pj[0] = 1.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { xj[a] = cv.x[(int64_t)j * DIM + a]; pj[1 + a] = sep_d(xi[a], xj[a], cv.periodic); }
      const double w = exp(nah2d * dist2_d<DIM>(xi, xj, cv.periodic));
      double r;
      if (linear) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < M; ++b) acc += z[b] * pj[b];
        r = w * acc;
      } else {
        r = w / wsum;
      }
      R[s] = (float)r;
    }
  }
}

int launch_stencils(const CaseView& cv, cudaStream_t s) {
  const int B = 128;
  const bool f64 = cv.storage == 0;
  if (cv.dim == 2) {
    if (f64) k_stencils<double, 2><<<grid_for(cv.n, B), B, 0, s>>>(cv);
    else k_stencils_f32<2><<<grid_for(cv.n, B), B, 0, s>>>(cv);
  } else {
    if (f64) k_stencils<double, 3><<<grid_for(cv.n, B), B, 0, s>>>(cv);
    else k_stencils_f32<3><<<grid_for(cv.n, B), B, 0, s>>>(cv);
  }
  return 1;
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
