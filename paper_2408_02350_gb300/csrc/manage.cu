// Point management (Sec. 3.5.2: removing and adding points), between steps.
//
// The paper names two operations: two points that come too close are replaced by
// one point at their midpoint, and points are added where the moving cloud opens
// holes; f at a new point is updated by least squares.  Readings (thresholds are
// not given): an interior point closer than rmin to a wall point is removed (the
// wall point stays on the boundary); remaining interior points i < j that are each
// other's nearest remaining interior neighbour and closer than rmin merge at the
// midpoint (the survivor keeps i's slot); an interior point in no merge with fewer than min_nbrs neighbours gets a
// new interior point at x_i - (h/2) c/|c|, c the sum of its neighbour separations,
// if that lies in [guard, 1 - guard]^dim (wrapped when periodic), outside the body's
// guard sphere (distance >= body_radius + guard from its centre) and no point of
// N(i) + {i} is within rmin of it.  f at a new position y is the linear WLS
// reconstruction at y from N(i) + {i}: p_k = (1, x_k - y), w_k = exp(-alpha
// |x_k - y|^2 / h^2), r_k = e_0^T (sum w p p^T)^-1 w_k p_k (the constant fit where
// fewer than dim + 1 points or a singular system).  Survivors keep their order;
// the added points follow in the order of the points that made them.
//
// Kernels: k_pm_wallnear, k_pm_nearest and k_pm_roles (one thread per point, FP64
// without fused multiply-add, so positions match a plain C evaluation bit for bit), k_pm_scan
// (one block: new indices of survivors and added points), k_pm_geom (new
// positions, kinds, normals), k_pm_rows (one CTA per point: copy or reconstruct
// rows of f), k_pm_lists (interior and wall index lists, wall map).
#include "bgk_internal.cuh"
#include "device_common.cuh"

namespace bgk {

namespace {

constexpr int PM_ROLE_KEEP = 0, PM_ROLE_MERGE = 1, PM_ROLE_GONE = 2, PM_ROLE_ADD = 3;

__device__ __forceinline__ double pm_dist2(const CaseView& cv, int i, int j) {
  double d2 = 0.0;
  for (int a = 0; a < cv.dim; ++a) {
    const double d = sep_d(cv.x[(int64_t)i * cv.dim + a], cv.x[(int64_t)j * cv.dim + a], cv.periodic);
    d2 = __dadd_rn(d2, __dmul_rn(d, d));
  }
  return d2;
}

// role[i] = GONE for an interior point closer than rmin to a wall point, KEEP otherwise.
__global__ void k_pm_wallnear(CaseView cv, double rmin2, int32_t* role) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  int r = PM_ROLE_KEEP;
  if (cv.kind[i] == 0) {
    for (int s = 0; s < cv.cnt[i]; ++s) {
      const int j = cv.col[(int64_t)i * cv.cap + s];
      if (cv.kind[j] != 0 && pm_dist2(cv, i, j) < rmin2) {
        r = PM_ROLE_GONE;
        break;
      }
    }
  }
  role[i] = r;
}

// Nearest remaining interior neighbour closer than rmin (-1: none, or i is removed).
__global__ void k_pm_nearest(CaseView cv, double rmin2, const int32_t* role, int32_t* nn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  int best_j = -1;
  double best = 0.0;
  if (cv.kind[i] == 0 && role[i] != PM_ROLE_GONE) {
    const int dim = cv.dim;
    for (int s = 0; s < cv.cnt[i]; ++s) {
      const int j = cv.col[(int64_t)i * cv.cap + s];
      if (cv.kind[j] != 0 || role[j] == PM_ROLE_GONE) continue;
      double d2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double d = sep_d(cv.x[(int64_t)i * dim + a], cv.x[(int64_t)j * dim + a], cv.periodic);
        d2 = __dadd_rn(d2, __dmul_rn(d, d));
      }
      if (best_j < 0 || d2 < best) { best_j = j; best = d2; }
    }
    if (best_j >= 0 && !(best < rmin2)) best_j = -1;
  }
  nn[i] = best_j;
}

__device__ __forceinline__ double wrap_unit(double y) {
  if (y >= 1.0) return __dadd_rn(y, -1.0);
  if (y < 0.0) return __dadd_rn(y, 1.0);
  return y;
}

__global__ void k_pm_roles(CaseView cv, const int32_t* nn, double rmin2, int min_nbrs, int32_t* role, double* ynew) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int dim = cv.dim, cap = cv.cap;
  int r = role[i];  // GONE: removed next to a wall
  const int j = nn[i];
  if (r == PM_ROLE_KEEP && j >= 0 && nn[j] == i) r = i < j ? PM_ROLE_MERGE : PM_ROLE_GONE;
  const int m = cv.cnt[i];
  if (r == PM_ROLE_KEEP && cv.kind[i] == 0 && m < min_nbrs && m > 0) {
    const double* xi = cv.x + (int64_t)i * dim;
    double c[3] = {0.0, 0.0, 0.0}, c2 = 0.0;
    for (int s = 0; s < m; ++s) {
      const double* xj = cv.x + (int64_t)cv.col[(int64_t)i * cap + s] * dim;
      for (int a = 0; a < dim; ++a) c[a] = __dadd_rn(c[a], sep_d(xi[a], xj[a], cv.periodic));
    }
    for (int a = 0; a < dim; ++a) c2 = __dadd_rn(c2, __dmul_rn(c[a], c[a]));
    if (c2 > 0.0) {
      const double cl = __dsqrt_rn(c2), step = __dmul_rn(0.5, cv.h);
      double y[3];
      bool ok = true;
      for (int a = 0; a < dim; ++a) {
        double ya = __dadd_rn(xi[a], -__dmul_rn(step, __ddiv_rn(c[a], cl)));
        if (cv.periodic) ya = wrap_unit(ya);
        else if (ya < cv.guard || ya > 1.0 - cv.guard) ok = false;
        y[a] = ya;
      }
      if (ok && cv.body) {
        // not inside the body's guard sphere
        double d2 = 0.0;
        for (int a = 0; a < dim; ++a) {
          const double d = __dadd_rn(cv.body->c[a], -y[a]);
          d2 = __dadd_rn(d2, __dmul_rn(d, d));
        }
        ok = !(d2 < __dmul_rn(cv.body_rg, cv.body_rg));
      }
      if (ok) {
        double d2 = 0.0;
        for (int a = 0; a < dim; ++a) {
          const double d = sep_d(y[a], xi[a], cv.periodic);
          d2 = __dadd_rn(d2, __dmul_rn(d, d));
        }
        ok = !(d2 < rmin2);
      }
      for (int s = 0; s < m && ok; ++s) {
        const double* xj = cv.x + (int64_t)cv.col[(int64_t)i * cap + s] * dim;
        double d2 = 0.0;
        for (int a = 0; a < dim; ++a) {
          const double d = sep_d(y[a], xj[a], cv.periodic);
          d2 = __dadd_rn(d2, __dmul_rn(d, d));
        }
        if (d2 < rmin2) ok = false;
      }
      if (ok) {
        r = PM_ROLE_ADD;
        for (int a = 0; a < dim; ++a) ynew[(int64_t)i * dim + a] = y[a];
      }
    }
  }
  role[i] = r;
}

// Exclusive scans (one block of 1024 threads, serial chunks per thread) of
// alive = role != GONE into newidx and of role == ADD into addidx; out[0] = survivors,
// out[1] = additions requested.
__global__ void k_pm_scan(int n, const int32_t* role, int32_t* newidx, int32_t* addidx, int32_t* out) {
  __shared__ int32_t s_w[2][32];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5;
  const int per = (n + T - 1) / T;
  const int lo = min(t * per, n), hi = min(lo + per, n);
  int32_t a = 0, b = 0;
  for (int i = lo; i < hi; ++i) { a += role[i] != PM_ROLE_GONE; b += role[i] == PM_ROLE_ADD; }
  int32_t xa = a, xb = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
    if (lane >= o) { xa += ya; xb += yb; }
  }
  if (lane == 31) { s_w[0][warp] = xa; s_w[1][warp] = xb; }
  __syncthreads();
  if (warp == 0) {
    int32_t va = lane < (T >> 5) ? s_w[0][lane] : 0, vb = lane < (T >> 5) ? s_w[1][lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t ya = __shfl_up_sync(0xffffffffu, va, o), yb = __shfl_up_sync(0xffffffffu, vb, o);
      if (lane >= o) { va += ya; vb += yb; }
    }
    s_w[0][lane] = va;
    s_w[1][lane] = vb;
  }
  __syncthreads();
  int32_t ra = xa - a + (warp > 0 ? s_w[0][warp - 1] : 0), rb = xb - b + (warp > 0 ? s_w[1][warp - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    newidx[i] = ra;
    addidx[i] = rb;
    ra += role[i] != PM_ROLE_GONE;
    rb += role[i] == PM_ROLE_ADD;
  }
  if (t == 0) { out[0] = s_w[0][31]; out[1] = s_w[1][31]; }
}

__global__ void k_pm_geom(CaseView cv, const int32_t* nn, const int32_t* role, const int32_t* newidx,
                          const int32_t* addidx, const int32_t* totals, int64_t cap_n, const double* ynew,
                          double* x2, int32_t* kind2, double* norm2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.n) return;
  const int dim = cv.dim, r = role[i];
  if (r == PM_ROLE_GONE) return;
  const int k = newidx[i];
  for (int a = 0; a < dim; ++a) {
    double y = cv.x[(int64_t)i * dim + a];
    if (r == PM_ROLE_MERGE) {
      const double xj = cv.x[(int64_t)nn[i] * dim + a];
      y = __dadd_rn(y, __dmul_rn(0.5, sep_d(y, xj, cv.periodic)));
      if (cv.periodic) y = wrap_unit(y);
    }
    x2[(int64_t)k * dim + a] = y;
    norm2[(int64_t)k * dim + a] = cv.normal[(int64_t)i * dim + a];
  }
  kind2[k] = cv.kind[i];
  if (r == PM_ROLE_ADD) {
    const int64_t ka = (int64_t)totals[0] + addidx[i];
    if (ka >= cap_n) return;
    for (int a = 0; a < dim; ++a) {
      x2[ka * dim + a] = ynew[(int64_t)i * dim + a];
      norm2[ka * dim + a] = 0.0;
    }
    kind2[ka] = 0;
  }
}

// Linear WLS reconstruction weights at y from the points src[0..m) (FP64,
// Gauss-Jordan with partial pivoting; the constant fit where m < dim + 1 or the
// system is singular).
__device__ void pm_weights(const CaseView& cv, const double* y, const int32_t* src, int m, double* r) {
  const int dim = cv.dim, mm = dim + 1;
  double a[4][8];
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 8; ++v) a[u][v] = 0.0;
  const double ih2 = 1.0 / (cv.h * cv.h);
  for (int s = 0; s < m; ++s) {
    const double* xk = cv.x + (int64_t)src[s] * dim;
    double pk[4] = {1.0, 0.0, 0.0, 0.0}, d2 = 0.0;
    for (int q = 0; q < dim; ++q) {
      pk[1 + q] = sep_d(y[q], xk[q], cv.periodic);
      d2 = __dadd_rn(d2, __dmul_rn(pk[1 + q], pk[1 + q]));
    }
    const double w = exp(-cv.alpha * d2 * ih2);
    for (int u = 0; u < mm; ++u)
      for (int v = 0; v < mm; ++v) a[u][v] += w * pk[u] * pk[v];
  }
  bool ok = m >= mm;
  double amax = 0.0;
  for (int u = 0; u < mm; ++u) {
    for (int v = 0; v < mm; ++v) amax = fmax(amax, fabs(a[u][v]));
    a[u][mm + u] = 1.0;
  }
  if (!(amax > 0.0)) ok = false;
  for (int c = 0; c < mm && ok; ++c) {
    int piv = c;
    for (int u = c + 1; u < mm; ++u)
      if (fabs(a[u][c]) > fabs(a[piv][c])) piv = u;
    if (!(fabs(a[piv][c]) > 1e-12 * amax)) { ok = false; break; }
    if (piv != c)
      for (int k = 0; k < 2 * mm; ++k) { const double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
    const double d = a[c][c];
    for (int k = 0; k < 2 * mm; ++k) a[c][k] /= d;
    for (int u = 0; u < mm; ++u) {
      if (u == c) continue;
      const double fct = a[u][c];
      for (int k = 0; k < 2 * mm; ++k) a[u][k] -= fct * a[c][k];
    }
  }
  double wsum = 0.0;
  for (int s = 0; s < m; ++s) {
    const double* xk = cv.x + (int64_t)src[s] * dim;
    double pk[4] = {1.0, 0.0, 0.0, 0.0}, d2 = 0.0;
    for (int q = 0; q < dim; ++q) {
      pk[1 + q] = sep_d(y[q], xk[q], cv.periodic);
      d2 = __dadd_rn(d2, __dmul_rn(pk[1 + q], pk[1 + q]));
    }
    const double w = exp(-cv.alpha * d2 * ih2);
    if (ok) {
      double acc = 0.0;
      for (int b = 0; b < mm; ++b) acc += a[0][mm + b] * pk[b];  // row 0 of the inverse (symmetric)
      r[s] = w * acc;
    } else {
      r[s] = w;
      wsum += w;
    }
  }
  if (!ok)
    for (int s = 0; s < m; ++s) r[s] /= wsum;
}

// One CTA per old point: copy its row of f to its new slot, or reconstruct it at the
// midpoint (merge survivor); an adding point also reconstructs the new point's row.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_pm_rows(CaseView cv, const int32_t* nn, const int32_t* role,
                                                 const int32_t* newidx, const int32_t* addidx, const int32_t* totals,
                                                 int64_t cap_n, const double* x2, const S* f, S* f2) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int i = blockIdx.x, r = role[i];
  if (r == PM_ROLE_GONE) return;
  const int64_t row = (int64_t)cv.ncomp * cv.NVp;
  const int cap = cv.cap, m = cv.cnt[i] + 1;
  int32_t* s_src = reinterpret_cast<int32_t*>(smem);
  double* s_r = reinterpret_cast<double*>(smem + sizeof(double) * ((cap + 2) / 2 + 1));
  const int64_t k = newidx[i];
  if (r != PM_ROLE_MERGE) {
    for (int64_t q = threadIdx.x; q < row; q += blockDim.x) f2[k * row + q] = f[(int64_t)i * row + q];
  }
  for (int pass = 0; pass < 2; ++pass) {
    // pass 0: the merge survivor at its midpoint; pass 1: the added point
    int64_t dst;
    if (pass == 0) {
      if (r != PM_ROLE_MERGE) continue;
      dst = k;
    } else {
      if (r != PM_ROLE_ADD) continue;
      dst = (int64_t)totals[0] + addidx[i];
      if (dst >= cap_n) continue;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_src[0] = i;
      for (int s = 1; s < m; ++s) s_src[s] = cv.col[(int64_t)i * cap + s - 1];
      pm_weights(cv, x2 + dst * cv.dim, s_src, m, s_r);
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < row; q += blockDim.x) {
      C acc = (C)0;
      for (int s = 0; s < m; ++s) acc += (C)s_r[s] * to_c(ld1(f + (int64_t)s_src[s] * row + q), (C)0);
      st1(f2 + dst * row + q, acc);
    }
  }
}

// Interior list: the old (Morton) order without the removed points, then the added
// points; wall list remapped; wall map rebuilt.  One block of 1024 threads (serial
// chunks per thread, block scan of the chunk counts).
__global__ void k_pm_lists(CaseView cv, const int32_t* role, const int32_t* newidx, const int32_t* addidx,
                           const int32_t* totals, int64_t cap_n, int32_t* int2, int32_t* wall_idx, int32_t* wall_of,
                           int64_t n_new) {
  __shared__ int32_t s_w[32];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5;
  const int nt = cv.n_int, per = (nt + T - 1) / T;
  const int lo = min(t * per, nt), hi = min(lo + per, nt);
  int32_t c = 0;
  for (int u = lo; u < hi; ++u) c += role[cv.int_idx[u]] != PM_ROLE_GONE;
  int32_t x = c;
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
  int32_t run = x - c + (warp > 0 ? s_w[warp - 1] : 0);
  for (int u = lo; u < hi; ++u) {
    const int i = cv.int_idx[u];
    if (role[i] != PM_ROLE_GONE) int2[run++] = newidx[i];
  }
  const int32_t base = s_w[31];
  for (int i = t; i < cv.n; i += T)
    if (role[i] == PM_ROLE_ADD && (int64_t)totals[0] + addidx[i] < cap_n) int2[base + addidx[i]] = totals[0] + addidx[i];
  for (int64_t i = t; i < n_new; i += T) wall_of[i] = -1;
  __syncthreads();
  for (int w = t; w < cv.n_wall; w += T) {
    const int nw = newidx[wall_idx[w]];
    wall_idx[w] = nw;
    wall_of[nw] = w;
  }
}

}  // namespace

int launch_manage_plan(const CaseView& cv, double rmin, int min_nbrs, int32_t* nn, int32_t* role, double* ynew,
                       int32_t* newidx, int32_t* addidx, int32_t* totals, cudaStream_t s) {
  const int B = 256, g = (cv.n + B - 1) / B;
  k_pm_wallnear<<<g, B, 0, s>>>(cv, rmin * rmin, role);
  k_pm_nearest<<<g, B, 0, s>>>(cv, rmin * rmin, role, nn);
  k_pm_roles<<<g, B, 0, s>>>(cv, nn, rmin * rmin, min_nbrs, role, ynew);
  k_pm_scan<<<1, 1024, 0, s>>>(cv.n, role, newidx, addidx, totals);
  return 4;
}

int launch_manage_apply(const CaseView& cv, int64_t cap_n, const int32_t* nn, const int32_t* role,
                        const double* ynew, const int32_t* newidx, const int32_t* addidx, const int32_t* totals,
                        double* x2, int32_t* kind2, double* norm2, const void* f, void* f2, int32_t* int2,
                        int32_t* wall_idx, int32_t* wall_of, int64_t n_new, cudaStream_t s) {
  const int B = 256, g = (cv.n + B - 1) / B;
  k_pm_geom<<<g, B, 0, s>>>(cv, nn, role, newidx, addidx, totals, cap_n, ynew, x2, kind2, norm2);
  const size_t smem = sizeof(double) * ((cv.cap + 2) / 2 + 1) + sizeof(double) * (cv.cap + 1);
  if (cv.storage == 0)
    k_pm_rows<double, double><<<cv.n, B, smem, s>>>(cv, nn, role, newidx, addidx, totals, cap_n, x2,
                                                    (const double*)f, (double*)f2);
  else if (cv.storage == 1)
    k_pm_rows<float, float><<<cv.n, B, smem, s>>>(cv, nn, role, newidx, addidx, totals, cap_n, x2,
                                                  (const float*)f, (float*)f2);
  else
    k_pm_rows<__nv_bfloat16, float><<<cv.n, B, smem, s>>>(cv, nn, role, newidx, addidx, totals, cap_n, x2,
                                                          (const __nv_bfloat16*)f, (__nv_bfloat16*)f2);
  k_pm_lists<<<1, 1024, 0, s>>>(cv, role, newidx, addidx, totals, cap_n, int2, wall_idx, wall_of, n_new);
  return 3;
}

}  // namespace bgk
