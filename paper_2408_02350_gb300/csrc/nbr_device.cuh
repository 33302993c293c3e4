// Per-point bodies of the cell-list neighbour search (Sec. 3.5.1, Sec. 4.2),
// shared by the separate kernels and the fused side-chain kernel.
#pragma once

#include "bgk_internal.cuh"
#include "device_common.cuh"

namespace bgk {

// Cell of point i (cells of side >= the search radius, x = 1 clamped to the last
// cell), its count, and the FP32 hi/lo split of x_i.
__device__ __forceinline__ void cell_assign_point(const CaseView& cv, const int i) {
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

// Exclusive scan of the cell counts into cell_start (one block of up to 1024 threads:
// per-thread serial sums, warp-shuffle scans, one scan of the warp totals), then
// clear the counts for k_cell_fill.
__device__ __forceinline__ void cell_scan_block(const CaseView& cv) {
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

__device__ __forceinline__ void cell_fill_point(const CaseView& cv, const int i) {
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
__device__ __forceinline__ void nbr_warp_point(const CaseView& cv, const int i, const int lane, int32_t* buf,
                                               const float lo, const float hi) {
  const int cap = CAND ? cv.ccap : cv.cap, nc = cv.nc;
  float xif[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xif[a] = cv.xf[(int64_t)i * DIM + a];
  const double h2 = cv.h2;
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
            j = checked_index(cv.cell_pts[q], cv.n, i, cv.status);
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
__device__ __forceinline__ void filter_warp_point(const CaseView& cv, const int i, const int lane, const float lo,
                                                  const float hi) {
  const int cap = cv.cap, nc = cv.ccnt[i];
  const int32_t* cand = cv.ccol + (int64_t)i * cv.ccap;
  int32_t* row = cv.col + (int64_t)i * cap;
  float xif[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xif[a] = cv.xf[(int64_t)i * DIM + a];
  const double h2 = cv.h2;
  int m = 0;
  for (int qb = 0; qb < nc; qb += 32) {
    const int q = qb + lane;
    bool inside = false;
    int j = -1;
    if (q < nc) {
      j = checked_index(cand[q], cv.n, i, cv.status);
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

// The exact test of filter_warp_point with a group of 4 lanes per point, 8 points per
// warp (group g = lane / 4 takes point i when valid), so that the candidate and
// position loads of 8 points and of 8 candidates per lane are in flight together.
// Candidates are taken in list order in chunks of 4 (one per lane of the group) and
// compacted in order with the group's bits of a warp ballot, so the rows equal
// filter_warp_point's.  Every lane of the warp calls it.
template <int DIM>
__device__ __forceinline__ void filter_group_point(const CaseView& cv, const int i, const bool valid, const int lane,
                                                   const float lo, const float hi) {
  constexpr int U = 8;  // chunks of 4 candidates per trip
  const int g = lane >> 2, sub = lane & 3;
  const int cap = cv.cap;
  const int nc = valid ? cv.ccnt[i] : 0;
  const int32_t* cand = cv.ccol + (int64_t)i * cv.ccap;
  int32_t* row = cv.col + (int64_t)i * cap;
  float xif[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) xif[a] = valid ? cv.xf[(int64_t)i * DIM + a] : 0.0f;
  const double h2 = cv.h2;
  const int ncmax = __reduce_max_sync(0xffffffffu, nc);
  int m = 0;  // uniform within the group
  for (int qb = 0; qb < ncmax; qb += 4 * U) {
    int jj[U];
    float d2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = qb + 4 * u + sub;
      jj[u] = q < nc ? checked_index(cand[q], cv.n, -1, cv.status) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float d2f = 0.0f;
      if (jj[u] >= 0) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          float d = cv.xf[(int64_t)jj[u] * DIM + a] - xif[a];
          if (cv.periodic) d = d > 0.5f ? d - 1.0f : (d < -0.5f ? d + 1.0f : d);
          d2f = fmaf(d, d, d2f);
        }
      }
      d2[u] = d2f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool inside = false;
      const int j = jj[u];
      if (j >= 0 && d2[u] <= hi) {
        inside = d2[u] <= lo;
        if (!inside) {
          double xi[DIM], xj[DIM];
#pragma unroll
          for (int a = 0; a < DIM; ++a) { xi[a] = cv.x[(int64_t)i * DIM + a]; xj[a] = cv.x[(int64_t)j * DIM + a]; }
          inside = dist2_d<DIM>(xi, xj, cv.periodic) <= h2;
        }
      }
      const unsigned gb = (__ballot_sync(0xffffffffu, inside) >> (4 * g)) & 0xFu;
      if (inside) {
        const int pos = m + __popc(gb & ((1u << sub) - 1u));
        if (pos < cap) row[pos] = j;
      }
      m += __popc(gb);
    }
  }
  if (valid && sub == 0) {
    cv.cnt[i] = m < cap ? m : cap;
    if (m > cap) set_status(cv.status, ST_OVERFLOW);
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
// accumulates its share of the neighbours into the normal matrix A = sum w dr dr^T in
// FP64 (separations, weights and the terms w dr_a dr_b in FP32, which carry the inputs'
// own precision; the sums in FP64), the group reduces A in FP64 with shuffles, and the
// group's first lane solves the normal equations in FP64 (inverse by cofactors,
// Sec. 3.4.1: S = A^-1).
// S is then rounded to FP32, and all lanes write the FP32 coefficients of their
// neighbours.  Every lane of the warp calls it (shuffles over the full warp); lanes with
// valid = false only take part in the shuffles.
template <int DIM, int LPP>
__device__ __forceinline__ void stencil_grp_point(const CaseView& cv, const int i, const bool valid, const int sub) {
  constexpr int NA = DIM == 2 ? 3 : 6;  // unique entries of the symmetric A
  const int m = valid ? cv.cnt[i] : 0;
  const int cap = cv.cap;
  const int32_t* row = cv.col + (int64_t)i * cap;
  const float nah2 = cv.nah2_f;
  double A[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) A[q] = 0.0;
  for (int s = sub; s < m; s += LPP) {
    float dr[DIM];
    sep_hilo<DIM>(cv, i, row[s], dr);
    float r2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) r2 = fmaf(dr[a], dr[a], r2);
    const float w = expf(nah2 * r2);
    int q = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const float wa = w * dr[a];
#pragma unroll
      for (int b = a; b < DIM; ++b) { A[q] += (double)(wa * dr[b]); ++q; }
    }
  }
#pragma unroll
  for (int o = LPP / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int q = 0; q < NA; ++q) A[q] += __shfl_xor_sync(0xffffffffu, A[q], o);
  float Sf[NA];
  int ok = 1;
  if (sub == 0) {
    double det, S[NA], scale;
    if constexpr (DIM == 2) {
      scale = fmax(fabs(A[0]), fabs(A[2]));
      det = A[0] * A[2] - A[1] * A[1];
      S[0] = A[2]; S[1] = -A[1]; S[2] = A[0];
    } else {
      // A = [a0 a1 a2; a1 a3 a4; a2 a4 a5]
      scale = fmax(fabs(A[0]), fmax(fabs(A[3]), fabs(A[5])));
      S[0] = A[3] * A[5] - A[4] * A[4];
      S[1] = A[4] * A[2] - A[1] * A[5];
      S[2] = A[1] * A[4] - A[3] * A[2];
      det = A[0] * S[0] + A[1] * S[1] + A[2] * S[2];
      S[3] = A[0] * A[5] - A[2] * A[2];
      S[4] = A[1] * A[2] - A[0] * A[4];
      S[5] = A[0] * A[3] - A[1] * A[1];
    }
    const double sc = DIM == 2 ? scale * scale : scale * scale * scale;
    ok = valid && m >= DIM && fabs(det) > 1e-12 * sc && isfinite(det);
    const double rdet = 1.0 / det;
#pragma unroll
    for (int q = 0; q < NA; ++q) Sf[q] = (float)(S[q] * rdet);
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

}  // namespace bgk
