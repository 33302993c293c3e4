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

// With sk (ALE skin lists) the cell kernels run only in steps that rebuild the candidates.
__global__ void k_cell_assign(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
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
  for (int a = 0; a < cv.dim; ++a) {
    const double xa = cv.x[(int64_t)i * cv.dim + a];
    const float hi = (float)xa;
    cv.xf[(int64_t)i * cv.dim + a] = hi;
    if (cv.xlo) cv.xlo[(int64_t)i * cv.dim + a] = (float)(xa - (double)hi);
  }
}

// Exclusive scan of the cell counts into cell_start (one block of 1024 threads:
// per-thread serial sums, warp-shuffle scans, one scan of the warp totals), then
// clear the counts for k_cell_fill.
__global__ void k_cell_scan(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
  __shared__ int32_t s_w[32];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5;
  const int ncell = cv.ncell;
  const int per = (ncell + T - 1) / T;
  const int lo = min(t * per, ncell), hi = min(lo + per, ncell);
  int32_t s = 0;
  for (int c = lo; c < hi; ++c) s += cv.cell_cnt[c];
  int32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t v = lane < (T >> 5) ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    s_w[lane] = v;
  }
  __syncthreads();
  int32_t run = x - s + (warp > 0 ? s_w[warp - 1] : 0);
  for (int c = lo; c < hi; ++c) {
    cv.cell_start[c] = run;
    run += cv.cell_cnt[c];
    cv.cell_cnt[c] = 0;
  }
  if (t == 0) cv.cell_start[ncell] = s_w[31];
}

__global__ void k_cell_fill(CaseView cv, const SkinState* sk) {
  if (sk && !sk->rebuild) return;
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
//
// One warp per point: lanes test the candidates of each of the 3^dim cells in
// parallel, matches are compacted with a ballot into a per-warp shared buffer,
// and the row is written in ascending order by a rank sort (every index in a
// row is distinct, so the rank of an entry is the number of smaller entries).
//
// CAND: candidate lists of the skin (radius h (1 + skin) in hi, superset test
// d2_f <= hi, rows into ccol / ccnt, positions saved in xb), only in steps that
// rebuild them; the cell counts are left at zero for the next rebuild.
template <int DIM, bool CAND>
__global__ void __launch_bounds__(256) k_neighbours_warp(CaseView cv, float lo, float hi) {
  extern __shared__ int32_t s_buf[];  // [W][cap]
  if (CAND && !cv.sk->rebuild) return;
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * W + warp;
  if (i >= cv.n) return;  // whole warp leaves together
  const int cap = CAND ? cv.ccap : cv.cap, nc = cv.nc;
  int32_t* buf = s_buf + warp * cap;
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
  // cells along x are stored consecutively, so each (y, z) row of the 3^dim
  // neighbourhood is one or two contiguous ranges of cell_pts
  int xr[2][2], nxr = 0;
  {
    int cs[3];
    for (int w = 0; w < len[0]; ++w) cs[w] = lst[0][w];
    for (int a = 1; a < len[0]; ++a)
      for (int b = a; b > 0 && cs[b - 1] > cs[b]; --b) { int tmp = cs[b]; cs[b] = cs[b - 1]; cs[b - 1] = tmp; }
    for (int w = 0; w < len[0]; ++w) {
      if (nxr > 0 && cs[w] == xr[nxr - 1][1] + 1) xr[nxr - 1][1] = cs[w];
      else { xr[nxr][0] = cs[w]; xr[nxr][1] = cs[w]; ++nxr; }
    }
  }
  int m = 0;  // warp-uniform count of matches
  for (int u = 0; u < len[2]; ++u)
    for (int v = 0; v < len[1]; ++v)
      for (int r = 0; r < nxr; ++r) {
        int c0 = 0;
        if (DIM >= 2) c0 += lst[1][v] * nc;
        if (DIM >= 3) c0 += lst[2][u] * nc * nc;
        const int q0 = cv.cell_start[c0 + xr[r][0]], q1 = cv.cell_start[c0 + xr[r][1] + 1];
        for (int qb = q0; qb < q1; qb += 32) {
          const int q = qb + lane;
          bool inside = false;
          int j = -1;
          if (q < q1) {
            j = cv.cell_pts[q];
            if (j != i) {
              float d2f = 0.0f;
#pragma unroll
              for (int a = 0; a < DIM; ++a) {
                float d = cv.xf[(int64_t)j * DIM + a] - xif[a];
                if (cv.periodic) d = d > 0.5f ? d - 1.0f : (d < -0.5f ? d + 1.0f : d);
                d2f = fmaf(d, d, d2f);
              }
              if (CAND) {
                inside = d2f <= hi;
              } else if (d2f <= hi) {
                inside = d2f <= lo;
                if (!inside) {
                  double xi[DIM], xj[DIM];
#pragma unroll
                  for (int a = 0; a < DIM; ++a) { xi[a] = cv.x[(int64_t)i * DIM + a]; xj[a] = cv.x[(int64_t)j * DIM + a]; }
                  inside = dist2_d<DIM>(xi, xj, cv.periodic) <= h2;
                }
              }
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, inside);
          if (inside) {
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) buf[pos] = j;
          }
          m += __popc(bal);
        }
      }
  __syncwarp();
  const int mm = m < cap ? m : cap;
  int32_t* row = (CAND ? cv.ccol : cv.col) + (int64_t)i * cap;
  for (int e = lane; e < mm; e += 32) {
    const int v = buf[e];
    int rank = 0;
    for (int k = 0; k < mm; ++k) rank += buf[k] < v ? 1 : 0;
    row[rank] = v;
  }
  if (CAND) {
    if (lane < DIM) cv.xb[(int64_t)i * DIM + lane] = cv.x[(int64_t)i * DIM + lane];
    // cell counts back to zero for the next rebuild (only k_cell_fill read them)
    for (int c = i * 32 + lane; c < cv.ncell; c += cv.n * 32) cv.cell_cnt[c] = 0;
  }
  if (lane == 0) {
    (CAND ? cv.ccnt : cv.cnt)[i] = mm;
    if (m > cap) set_status(cv.status, ST_OVERFLOW);
  }
}

// The exact test of k_neighbours_warp applied to the candidate list of each point
// (ascending, so the kept entries are ascending too; one warp per point).  The
// candidates contain every point within h: a pair within h now was within
// h + 2 max|x - x_b| < h (1 + skin) at the build.
template <int DIM>
__global__ void __launch_bounds__(256) k_filter(CaseView cv, float lo, float hi) {
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * W + warp;
  if (i >= cv.n) return;
  const int cap = cv.cap, nc = cv.ccnt[i];
  const int32_t* cand = cv.ccol + (int64_t)i * cv.ccap;
  int32_t* row = cv.col + (int64_t)i * cap;
  float xif[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xif[a] = cv.xf[(int64_t)i * DIM + a];
  const double h2 = __dmul_rn(cv.h, cv.h);
  int m = 0;
  for (int qb = 0; qb < nc; qb += 32) {
    const int q = qb + lane;
    bool inside = false;
    int j = -1;
    if (q < nc) {
      j = cand[q];
      float d2f = 0.0f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float d = cv.xf[(int64_t)j * DIM + a] - xif[a];
        if (cv.periodic) d = d > 0.5f ? d - 1.0f : (d < -0.5f ? d + 1.0f : d);
        d2f = fmaf(d, d, d2f);
      }
      if (d2f <= hi) {
        inside = d2f <= lo;
        if (!inside) {
          double xi[DIM], xj[DIM];
#pragma unroll
          for (int a = 0; a < DIM; ++a) { xi[a] = cv.x[(int64_t)i * DIM + a]; xj[a] = cv.x[(int64_t)j * DIM + a]; }
          inside = dist2_d<DIM>(xi, xj, cv.periodic) <= h2;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, inside);
    if (inside) {
      const int pos = m + __popc(bal & ((1u << lane) - 1u));
      if (pos < cap) row[pos] = j;
    }
    m += __popc(bal);
  }
  if (lane == 0) {
    cv.cnt[i] = m < cap ? m : cap;
    if (m > cap) set_status(cv.status, ST_OVERFLOW);
  }
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

// Separation x_j - x_i from the FP32 hi/lo split of the positions: the
// difference of the high parts is exact or rounded once, the low parts add the
// remainder, so the result carries about 1e-7 relative error without any FP64
// arithmetic (minimum image on the high part for periodic boxes).
template <int DIM>
__device__ __forceinline__ void sep_hilo(const CaseView& cv, int i, int j, float (&dr)[DIM]) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    float dh = cv.xf[(int64_t)j * DIM + a] - cv.xf[(int64_t)i * DIM + a];
    if (cv.periodic) dh = dh > 0.5f ? dh - 1.0f : (dh < -0.5f ? dh + 1.0f : dh);
    dr[a] = dh + (cv.xlo[(int64_t)j * DIM + a] - cv.xlo[(int64_t)i * DIM + a]);
  }
}

// FP32/BF16 path, interior points: a group of LPP lanes per point.  Each lane
// accumulates its share of the neighbours into the normal matrix
// A = sum w dr dr^T (FP32), the group reduces A with shuffles, and the group's
// first lane inverts it in FP64; all lanes then write the FP32 coefficients of
// their neighbours.
template <int DIM, int LPP>
__global__ void __launch_bounds__(256) k_stencils_grp(CaseView cv) {
  constexpr int NA = DIM == 2 ? 3 : 6;  // unique entries of the symmetric A
  const int gid = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPP);
  const int sub = threadIdx.x % LPP;
  const bool valid = gid < cv.n_int;
  const int i = valid ? cv.int_idx[gid] : 0;
  const int m = valid ? cv.cnt[i] : 0;
  const int cap = cv.cap;
  const int32_t* row = cv.col + (int64_t)i * cap;
  const float nah2 = (float)(-cv.alpha / (cv.h * cv.h));
  float A[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) A[q] = 0.0f;
  for (int s = sub; s < m; s += LPP) {
    float dr[DIM];
    sep_hilo<DIM>(cv, i, row[s], dr);
    float r2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) r2 = fmaf(dr[a], dr[a], r2);
    const float w = expf(nah2 * r2);
    int q = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = a; b < DIM; ++b) { A[q] = fmaf(w * dr[a], dr[b], A[q]); ++q; }
  }
#pragma unroll
  for (int o = LPP / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int q = 0; q < NA; ++q) A[q] += __shfl_xor_sync(0xffffffffu, A[q], o);
  float Sf[NA];
  int ok = 1;
  if (sub == 0) {
    double Ad[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) Ad[q] = (double)A[q];
    double det, S[NA], scale;
    if constexpr (DIM == 2) {
      scale = fmax(fabs(Ad[0]), fabs(Ad[2]));
      det = Ad[0] * Ad[2] - Ad[1] * Ad[1];
      const double id = 1.0 / det;
      S[0] = Ad[2] * id; S[1] = -Ad[1] * id; S[2] = Ad[0] * id;
    } else {
      // A = [a0 a1 a2; a1 a3 a4; a2 a4 a5]
      scale = fmax(fabs(Ad[0]), fmax(fabs(Ad[3]), fabs(Ad[5])));
      const double c00 = Ad[3] * Ad[5] - Ad[4] * Ad[4];
      const double c01 = Ad[4] * Ad[2] - Ad[1] * Ad[5];
      const double c02 = Ad[1] * Ad[4] - Ad[3] * Ad[2];
      det = Ad[0] * c00 + Ad[1] * c01 + Ad[2] * c02;
      const double id = 1.0 / det;
      S[0] = c00 * id; S[1] = c01 * id; S[2] = c02 * id;
      S[3] = (Ad[0] * Ad[5] - Ad[2] * Ad[2]) * id;
      S[4] = (Ad[1] * Ad[2] - Ad[0] * Ad[4]) * id;
      S[5] = (Ad[0] * Ad[3] - Ad[1] * Ad[1]) * id;
    }
    const double sc = DIM == 2 ? scale * scale : scale * scale * scale;
    ok = valid && m >= DIM && fabs(det) > 1e-12 * sc && isfinite(det);
#pragma unroll
    for (int q = 0; q < NA; ++q) Sf[q] = (float)S[q];
  }
  const int src = (threadIdx.x & 31) & ~(LPP - 1);
#pragma unroll
  for (int q = 0; q < NA; ++q) Sf[q] = __shfl_sync(0xffffffffu, Sf[q], src);
  ok = __shfl_sync(0xffffffffu, ok, src);
  if (!valid) return;
  float* P = (float*)cv.P + (int64_t)i * cap * DIM * DIM;
  if (!ok) {
    if (sub == 0) set_status(cv.status, ST_SINGULAR);
    for (int s = sub; s < m * DIM * DIM; s += LPP) P[s] = 0.0f;
    return;
  }
  float S[DIM][DIM];
  if constexpr (DIM == 2) {
    S[0][0] = Sf[0]; S[0][1] = Sf[1]; S[1][0] = Sf[1]; S[1][1] = Sf[2];
  } else {
    S[0][0] = Sf[0]; S[0][1] = Sf[1]; S[0][2] = Sf[2];
    S[1][0] = Sf[1]; S[1][1] = Sf[3]; S[1][2] = Sf[4];
    S[2][0] = Sf[2]; S[2][1] = Sf[4]; S[2][2] = Sf[5];
  }
  for (int s = sub; s < m; s += LPP) {
    float dr[DIM];
    sep_hilo<DIM>(cv, i, row[s], dr);
    float r2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) r2 = fmaf(dr[a], dr[a], r2);
    const float w = expf(nah2 * r2);
    float coef[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      float acc = 0.0f;
#pragma unroll
      for (int b = 0; b < DIM; ++b) acc = fmaf(S[a][b], dr[b], acc);
      coef[a] = w * acc;
    }
    const float rinv = rsqrtf(r2);
    float E[DIM][DIM];
    if constexpr (DIM == 2) {
      const float nx = dr[0] * rinv, ny = dr[1] * rinv;
      E[0][0] = nx; E[0][1] = ny;
      E[1][0] = -ny; E[1][1] = nx;
    } else {
      const float rxy2 = dr[0] * dr[0] + dr[1] * dr[1];
      const float rxyinv = rxy2 > 0.0f ? rsqrtf(rxy2) : 0.0f;
      const float cphi = rxy2 > 0.0f ? dr[0] * rxyinv : 1.0f, sphi = rxy2 > 0.0f ? dr[1] * rxyinv : 0.0f;
      const float cth = dr[2] * rinv, sth = rxy2 * rxyinv * rinv;
      E[0][0] = dr[0] * rinv; E[0][1] = dr[1] * rinv; E[0][2] = cth;
      E[1][0] = cth * cphi; E[1][1] = cth * sphi; E[1][2] = -sth;
      E[2][0] = -sphi; E[2][1] = cphi; E[2][2] = 0.0f;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      float ab = 0.0f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) ab = fmaf(E[d][a], coef[a], ab);
#pragma unroll
      for (int a = 0; a < DIM; ++a) P[(s * DIM + d) * DIM + a] = ab * E[d][a];
    }
  }
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
  const float nah2 = (float)(-cv.alpha / (cv.h * cv.h));
  const float inv_h = (float)(1.0 / cv.h);  // basis (1, dr/h): same weights, O(1) matrix entries
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
  if (f64) {
    if (part == 2) return 0;
    if (cv.dim == 2) k_stencils<double, 2><<<grid_for(cv.n, B), B, 0, s>>>(cv);
    else k_stencils<double, 3><<<grid_for(cv.n, B), B, 0, s>>>(cv);
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
