// Point motion of one step (Eqs. originalALE1, ALE1), shared by the motion kernel
// and the fused side-chain kernel: FP64 without fused multiply-add, so positions
// match a plain C evaluation of x + dt*U bit for bit.
#pragma once

#include "bgk_internal.cuh"
#include "device_common.cuh"

namespace bgk {

// Stores the new position y of point i; with skin lists also the FP32 split of y
// (the prefilters read it; k_cell_assign sets it only when the cells are rebuilt),
// and returns the squared displacement since the candidate build.
__device__ __forceinline__ double store_position(const CaseView& cv, const int i, const double* y) {
  double d2 = 0.0;
  for (int a = 0; a < cv.dim; ++a) {
    cv.x[(int64_t)i * cv.dim + a] = y[a];
    if (cv.sk) {
      const float hi = (float)y[a];
      cv.xf[(int64_t)i * cv.dim + a] = hi;
      cv.xlo[(int64_t)i * cv.dim + a] = (float)(y[a] - (double)hi);
      const double d = __dadd_rn(y[a], -cv.xb[(int64_t)i * cv.dim + a]);
      d2 = __dadd_rn(d2, __dmul_rn(d, d));
    }
  }
  return d2;
}

// x_i += dt U_i^{n+1} for one interior point (FP64 without fused multiply-add),
// clamped to [guard, 1 - guard] or wrapped in a periodic box.  With a body (cn =
// its centre after this step, else null), a point that ends closer than body_rg to
// cn is put back on that sphere along the ray from cn (at cn + body_rg e_x if it
// sits on cn).  Every clamp is counted.
__device__ __forceinline__ double move_point(const CaseView& cv, const int i, const double* cn) {
  unsigned long long nclamp = 0;
  double y[3];
  for (int a = 0; a < cv.dim; ++a) {
    double ya = __dadd_rn(cv.x[(int64_t)i * cv.dim + a], __dmul_rn(cv.dt, cv.mom[(int64_t)i * MOM_STRIDE + 1 + a]));
    if (cv.periodic) {
      if (ya >= 1.0) ya = __dadd_rn(ya, -1.0);
      else if (ya < 0.0) ya = __dadd_rn(ya, 1.0);
    } else if (ya < cv.guard) { ya = cv.guard; ++nclamp; }
    else if (ya > 1.0 - cv.guard) { ya = 1.0 - cv.guard; ++nclamp; }
    y[a] = ya;
  }
  if (cn) {
    double d[3], r2 = 0.0;
    for (int a = 0; a < cv.dim; ++a) {
      d[a] = __dadd_rn(y[a], -cn[a]);
      r2 = __dadd_rn(r2, __dmul_rn(d[a], d[a]));
    }
    const double rg = cv.body_rg;
    if (r2 < __dmul_rn(rg, rg)) {
      if (r2 > 0.0) {
        const double sc = __ddiv_rn(rg, __dsqrt_rn(r2));
        for (int a = 0; a < cv.dim; ++a) y[a] = __dadd_rn(cn[a], __dmul_rn(d[a], sc));
      } else {
        for (int a = 0; a < cv.dim; ++a) y[a] = __dadd_rn(cn[a], a == 0 ? rg : 0.0);
      }
      ++nclamp;
    }
  }
  if (nclamp) atomicAdd(&cv.status->clamps, nclamp);
  return store_position(cv, i, y);
}

// A boundary point of the body: x_b += dt body_u.
__device__ __forceinline__ double move_body_point(const CaseView& cv, const int b) {
  double y[3];
  for (int a = 0; a < cv.dim; ++a) y[a] = __dadd_rn(cv.x[(int64_t)b * cv.dim + a], __dmul_rn(cv.dt, cv.body_u[a]));
  return store_position(cv, b, y);
}

// The body's centre after this step, c + dt body_u (every thread forms the same value).
__device__ __forceinline__ void body_centre_next(const CaseView& cv, double* cn) {
  for (int a = 0; a < 3; ++a) cn[a] = 0.0;
  if (cv.body)
    for (int a = 0; a < cv.dim; ++a) cn[a] = __dadd_rn(cv.body->c[a], __dmul_rn(cv.dt, cv.body_u[a]));
}

// Motion thread t: t < n_int moves interior point int_idx[t]; with a body, threads
// [n_int, n_int + n_wall) move the body's boundary points among the wall points.
// Returns the squared displacement since the candidate build (0 without skin lists).
__device__ __forceinline__ double move_thread(const CaseView& cv, const int t, const double* cn) {
  if (t < cv.n_int) return move_point(cv, cv.int_idx[t], cv.body ? cn : nullptr);
  if (cv.body && t < cv.n_int + cv.n_wall) {
    const int b = cv.wall_idx[t - cv.n_int];
    if (cv.kind[b] == cv.body_wall) return move_body_point(cv, b);
  }
  return 0.0;
}

}  // namespace bgk
