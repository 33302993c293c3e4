// Warp-per-point transport + moments + relaxation in FP32 arithmetic (FP32 or BF16
// storage), Sec. 3.2 and 3.4: the per-point body and its pieces, shared by the
// single-case and batched transport kernels.
#pragma once

#include "bgk_internal.cuh"
#include "device_common.cuh"

namespace bgk {

// Neighbour rows whose loads the compiler may overlap (unroll of the neighbour loop).
#ifndef BGK_NBR_UNROLL
#define BGK_NBR_UNROLL 2
#endif
constexpr int kNbrUnroll = BGK_NBR_UNROLL;

// ---------------------------------------------------------------------------
// transport + moments + relaxation, FP32 arithmetic (FP32 or BF16 storage):
// one warp per interior point.  Each lane owns 4 consecutive velocities of
// every 128-velocity slice; the warps of a CTA handle consecutive points, whose
// shared neighbour rows are often served from L1.  f~ of
// a slice is written to the output row and re-read after the moments, which are
// warp-shuffle sums of per-lane Kahan-compensated slice sums (no CTA barrier).
// With ROW4 (nv % 4 == 0) a lane's 4 velocities share (v_y, v_z), so the
// projection c.P_d costs one FMA per velocity: c.P_d = c_x P_dx + (c_y P_dy + c_z P_dz).
// ---------------------------------------------------------------------------
// Quotient k / n for 0 <= k < 2^13, 1 <= n <= 64 by a float reciprocal: (k + 1/2)/n lies at least
// 1/(2n) away from an integer and the float error is below (k/n + 1) 2^-23, so truncation is exact.
__device__ __forceinline__ int fdiv_small(int k, float inv_n) { return (int)(((float)k + 0.5f) * inv_n); }

// Velocity components of the VPL velocities k0..k0+VPL-1.  With ROW (nv % VPL == 0,
// k0 % VPL == 0) they share every component but the first.
template <int DIM, int VPL, bool ROW>
__device__ __forceinline__ void chunk_velocities(int k0, int nv, int NV, float inv_nv, const float* s_v,
                                                 float (&vel)[VPL][DIM], bool (&kin)[VPL]) {
  if (ROW) {
    int q = fdiv_small(k0, inv_nv);
    const int kx0 = k0 - q * nv;
    if constexpr (VPL % 4 == 0) {
      // kx0 is a multiple of VPL (k0 and nv are), so the first components come in
      // aligned groups of four
#pragma unroll
      for (int e = 0; e < VPL; e += 4) {
        const float4 x = *reinterpret_cast<const float4*>(s_v + kx0 + e);
        vel[e][0] = x.x; vel[e + 1][0] = x.y; vel[e + 2][0] = x.z; vel[e + 3][0] = x.w;
      }
#pragma unroll
      for (int e = 0; e < VPL; ++e) kin[e] = k0 + e < NV;
    } else {
#pragma unroll
      for (int e = 0; e < VPL; ++e) { vel[e][0] = s_v[kx0 + e]; kin[e] = k0 + e < NV; }
    }
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
      const int q2 = fdiv_small(q, inv_nv);
      const float va = s_v[q - q2 * nv];
      q = q2;
#pragma unroll
      for (int e = 0; e < VPL; ++e) vel[e][a] = va;
    }
  } else {
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
      int kk = k0 + e;
      kin[e] = kk < NV;
      if (!kin[e]) kk = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int q = fdiv_small(kk, inv_nv);
        vel[e][a] = s_v[kk - q * nv];
        kk = q;
      }
    }
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// 2^x by the hardware's approximate base-2 exponential (relative error about 2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 min0(float2 p) { return make_float2(fminf(p.x, 0.0f), fminf(p.y, 0.0f)); }

template <typename S, int VPL>
__device__ __forceinline__ void ldv(const S* p, float (&v)[VPL]) {
#pragma unroll
  for (int q = 0; q < VPL / 4; ++q) ld4(p + 4 * q, v + 4 * q);
}
// Neighbour rows of f^n through the read-only data path (f^n is not written while
// the transport runs: the output goes to the other buffer).
__device__ __forceinline__ void ld4_ro(const float* p, float v[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4_ro(const __nv_bfloat16* p, float v[4]) {
  uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
  const float2 l = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&a.x));
  const float2 h = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&a.y));
  v[0] = l.x; v[1] = l.y; v[2] = h.x; v[3] = h.y;
}
template <typename S, int VPL>
__device__ __forceinline__ void ldv_ro(const S* p, float (&v)[VPL]) {
#pragma unroll
  for (int q = 0; q < VPL / 4; ++q) ld4_ro(p + 4 * q, v + 4 * q);
}
template <typename S, int VPL>
__device__ __forceinline__ void stv(S* p, const float (&v)[VPL]) {
#pragma unroll
  for (int q = 0; q < VPL / 4; ++q) st4(p + 4 * q, v + 4 * q);
}

// Upwind sums of one neighbour row for the VPL = 2 NP velocities of a lane that lie
// in one row of the velocity grid (they share every component but the first):
//   m = sum_d min(c.P_d, 0),  sk += m,  acc_c += m f_j,c
// in packed FP32x2 arithmetic, with c.P_d = c_x P_dx + (c_y P_dy + c_z P_dz).
template <int DIM, int NC, int NP>
__device__ __forceinline__ void row_upwind(const float2 (&cx)[NP], const float (&crest)[DIM - 1],
                                           const float (&P)[DIM * DIM], const float (&fv)[NC][2 * NP],
                                           float2 (&skp)[NP], float2 (&ap)[NC][NP]) {
  float2 mk[NP];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float b = crest[0] * P[d * DIM + 1];
#pragma unroll
    for (int a = 2; a < DIM; ++a) b = fmaf(crest[a - 1], P[d * DIM + a], b);
    const float2 px = f2(P[d * DIM], P[d * DIM]), bb = f2(b, b);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float2 mq = min0(__ffma2_rn(cx[q], px, bb));
      mk[q] = d == 0 ? mq : __fadd2_rn(mk[q], mq);
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    skp[q] = __fadd2_rn(skp[q], mk[q]);
#pragma unroll
    for (int c = 0; c < NC; ++c) ap[c][q] = __ffma2_rn(mk[q], f2(fv[c][2 * q], fv[c][2 * q + 1]), ap[c][q]);
  }
}

// a - b in packed FP32x2 with one rounding per half (b times -1 is exact), as a scalar
// subtraction rounds.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f, -1.0f), a); }

// Compensated (Kahan) addition of the slice sums ps to the running sums, two at a time
// in packed FP32x2 (each half rounds as the scalar form would).
template <int N>
__device__ __forceinline__ void kahan_add(const float (&ps)[N], float (&msum)[N], float (&mcmp)[N]) {
#pragma unroll
  for (int q = 0; q + 1 < N; q += 2) {
    const float2 y = sub2(f2(ps[q], ps[q + 1]), f2(mcmp[q], mcmp[q + 1]));
    const float2 m = f2(msum[q], msum[q + 1]);
    const float2 t = __fadd2_rn(m, y);
    const float2 c = sub2(sub2(t, m), y);
    msum[q] = t.x; msum[q + 1] = t.y;
    mcmp[q] = c.x; mcmp[q + 1] = c.y;
  }
  if (N % 2) {
    const float y = ps[N - 1] - mcmp[N - 1];
    const float t = msum[N - 1] + y;
    mcmp[N - 1] = (t - msum[N - 1]) - y;
    msum[N - 1] = t;
  }
}

// End of a velocity slice: f~ = f_i - 2 dt (acc - sk f_i) for the lane's VPL
// velocities, written to the output row (and to the adjoint's tape when one is
// attached); the slice's moment sums are Kahan-added to the lane's running sums.
// AVG (second stage of the two-stage transport): f~ = (f_avg,i + f~) / 2, f_avg the
// state at the start of the step, whose row i is read before the output overwrites it.
// ROW: the lane's velocities share every component but the first (then the sums of
// v_a g for a >= 1 are v_a sum g), and f~ is formed in packed FP32x2 pairs.
template <typename S, int DIM, int NC, int VPL, bool AVG = false, bool ROW = false>
__device__ __forceinline__ void slice_out(const CaseView& cv, const int i, const int k0, const float (&vel)[VPL][DIM],
                                          const bool (&kin)[VPL], const float (&acc)[NC][VPL],
                                          const float (&sk)[VPL], const float two_dt, float (&msum)[DIM + 2],
                                          float (&mcmp)[DIM + 2]) {
  const int NVp = cv.NVp;
  const int64_t rowlen = (int64_t)NC * NVp;
  const S* fi = reinterpret_cast<const S*>(cv.f_in) + (int64_t)i * rowlen;
  S* fo = reinterpret_cast<S*>(cv.f_out) + (int64_t)i * rowlen;
  float fiv[NC][VPL], ft[NC][VPL], fav[NC][AVG ? VPL : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) ldv<S, VPL>(fi + (int64_t)c * NVp + k0, fiv[c]);
  if constexpr (AVG) {
    const S* fa = reinterpret_cast<const S*>(cv.f_avg) + (int64_t)i * rowlen;
#pragma unroll
    for (int c = 0; c < NC; ++c) ldv<S, VPL>(fa + (int64_t)c * NVp + k0, fav[c]);
  }
  float ps[DIM + 2];
  if constexpr (ROW && VPL % 2 == 0) {
    constexpr int NP = VPL / 2;
    const float2 ntd = f2(-two_dt, -two_dt);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float2 nsk = __fmul2_rn(f2(sk[2 * q], sk[2 * q + 1]), f2(-1.0f, -1.0f));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 fq = f2(fiv[c][2 * q], fiv[c][2 * q + 1]);
        const float2 t = __ffma2_rn(nsk, fq, f2(acc[c][2 * q], acc[c][2 * q + 1]));  // acc - sk f_i
        float2 r = __ffma2_rn(ntd, t, fq);                                              // f_i - 2 dt (.)
        if (AVG) r = __fmul2_rn(f2(0.5f, 0.5f), __fadd2_rn(r, f2(fav[c][2 * q], fav[c][2 * q + 1])));
        ft[c][2 * q] = r.x; ft[c][2 * q + 1] = r.y;
      }
    }
    if (!kin[VPL - 1]) {
#pragma unroll
      for (int e = 0; e < VPL; ++e)
#pragma unroll
        for (int c = 0; c < NC; ++c) ft[c][e] = kin[e] ? ft[c][e] : 0.0f;
    }
    // sum g, sum v_x g, sum |v|^2 g (+ sum h) in pairs; |v|^2 = v_x^2 + r2
    float r2 = 0.0f;
#pragma unroll
    for (int a = 1; a < DIM; ++a) r2 = fmaf(vel[0][a], vel[0][a], r2);
    float2 gs = f2(0.0f, 0.0f), xg = gs, wg = gs, hs = gs;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float2 g = f2(ft[0][2 * q], ft[0][2 * q + 1]);
      const float2 vx = f2(vel[2 * q][0], vel[2 * q + 1][0]);
      gs = __fadd2_rn(gs, g);
      xg = __ffma2_rn(vx, g, xg);
      wg = __ffma2_rn(__ffma2_rn(vx, vx, f2(r2, r2)), g, wg);
      if (NC == 2) hs = __fadd2_rn(hs, f2(ft[NC - 1][2 * q], ft[NC - 1][2 * q + 1]));
    }
    ps[0] = gs.x + gs.y;
    ps[1] = xg.x + xg.y;
#pragma unroll
    for (int a = 1; a < DIM; ++a) ps[1 + a] = vel[0][a] * ps[0];
    ps[DIM + 1] = NC == 2 ? (wg.x + wg.y) + (hs.x + hs.y) : wg.x + wg.y;
  } else {
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) ps[q] = 0.0f;
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
#pragma unroll
      for (int c = 0; c < NC; ++c) ft[c][e] = kin[e] ? fiv[c][e] - two_dt * (acc[c][e] - sk[e] * fiv[c][e]) : 0.0f;
      if (AVG) {
#pragma unroll
        for (int c = 0; c < NC; ++c) ft[c][e] = 0.5f * (ft[c][e] + fav[c][e]);
      }
      const float g = ft[0][e];
      float v2 = 0.0f;
      ps[0] += g;
#pragma unroll
      for (int a = 0; a < DIM; ++a) { ps[1 + a] = fmaf(vel[e][a], g, ps[1 + a]); v2 = fmaf(vel[e][a], vel[e][a], v2); }
      ps[DIM + 1] = fmaf(v2, g, ps[DIM + 1]);
      if (NC == 2) ps[DIM + 1] += ft[NC - 1][e];
    }
  }
  kahan_add<DIM + 2>(ps, msum, mcmp);
#pragma unroll
  for (int c = 0; c < NC; ++c) stv<S, VPL>(fo + (int64_t)c * NVp + k0, ft[c]);
  if (cv.ft_out) {
#pragma unroll
    for (int c = 0; c < NC; ++c) stv<float, VPL>(cv.ft_out + (int64_t)i * rowlen + (int64_t)c * NVp + k0, ft[c]);
    stv<float, VPL>(cv.sk_out + (int64_t)i * NVp + k0, sk);
  }
}

// Moments of f~_i from the raw sums tot = (sum g, sum v g, sum |v|^2 g (+ sum h)) in
// FP64 (U = sum v g / R and T = (sum |v|^2 g - R |U|^2) / (3 R), where the difference
// cancels), tau and the Maxwellian in FP32 from them, then the relaxation pass over the
// output row: f^{n+1} = (tau f~ + dt M)/(tau + dt) (RK = 1: the exact relaxation over
// dt/2).  All 32 lanes of the warp take part, each with the same tot.  SH: the row holds
// the velocity slab that starts at cv.vk0.
template <typename S, int DIM, bool ROW, int VPL, bool SH = false, int RK = 0>
__device__ __forceinline__ void relax_point(const CaseView& cv, const int i, const float* s_v,
                                            const double (&tot)[DIM + 2]) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  const int lane = threadIdx.x & 31;
  const int nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int vk0 = SH ? cv.vk0 : 0;
  const float inv_nv = 1.0f / (float)nv;
  const int nchunk = NVp / VPL;
  const int nslice = (nchunk + 31) >> 5;
  S* fo = reinterpret_cast<S*>(cv.f_out) + (int64_t)i * NC * NVp;
  const double R = tot[0], rR = 1.0 / R;
  double Ud[DIM], u2d = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) { Ud[a] = tot[1 + a] * rR; u2d = fma(Ud[a], Ud[a], u2d); }
  const double Td = fma(-R, u2d, tot[DIM + 1]) * rR * (1.0 / 3.0);
  const double rhod = R * cv.wv;
  float Un[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) Un[a] = (float)Ud[a];
  const float Tn = (float)Td, rho = (float)rhod;
  if (lane == 0) {
    double* mo = cv.mom + (int64_t)i * MOM_STRIDE;
    mo[0] = rhod;
#pragma unroll
    for (int a = 0; a < 3; ++a) mo[1 + a] = a < DIM ? Ud[a < DIM ? a : 0] : 0.0;
    mo[4] = Td;
    // (non-positive or non-finite values stay so in FP32)
    if (!(rho > 0.0f) || !(Tn > 0.0f) || !isfinite(rho) || !isfinite(Tn)) set_status(cv.status, ST_NONFINITE);
  }
  float ca = 1.0f, cb = 0.0f, pref = 0.0f, nl2 = 0.0f;
  if (cv.tau_mode != 2 && rho > 0.0f && Tn > 0.0f) {
    const float kn = cv.kn_f, dtf = cv.dt_f;
    const float tau = cv.tau_mode == 1 ? 0.7978845608f * kn : 0.7978845608f * kn / (rho * sqrtf(Tn));
    if (RK == 1) {
      // exact relaxation over dt/2 (the second-order step): f = e f + (1 - e) M, e = exp(-dt/(2 tau))
      ca = expf(-0.5f * dtf / tau);
      cb = -expm1f(-0.5f * dtf / tau);
    } else {
      ca = tau / (tau + dtf);
      cb = dtf / (tau + dtf);
    }
    const float twopiT = 6.283185307f * Tn;
    pref = cb * (DIM == 2 ? rho / twopiT : rho / (twopiT * sqrtf(twopiT)));
    nl2 = -0.5f / Tn;
  }
  const float l2 = nl2 * 1.44269504f;  // log2(e)
  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = VPL * chunk;
    float vel[VPL][DIM];
    bool kin[VPL];
    chunk_velocities<DIM, VPL, ROW>(k0 + vk0, nv, NV + vk0, inv_nv, s_v, vel, kin);
    float ft[NC][VPL], out[NC][VPL];
#pragma unroll
    for (int c = 0; c < NC; ++c) ldv<S, VPL>(fo + (int64_t)c * NVp + k0, ft[c]);
    if constexpr (ROW && VPL % 2 == 0) {
      // in packed pairs: |v - U|^2 = (v_x - U_x)^2 + r2, r2 shared by the lane's velocities;
      // M from 2^(l2 |v - U|^2), l2 = -log2(e) / (2 T)
      float r2 = 0.0f;
#pragma unroll
      for (int a = 1; a < DIM; ++a) {
        const float d = vel[0][a] - Un[a];
        r2 = fmaf(d, d, r2);
      }
#pragma unroll
      for (int q = 0; q < VPL / 2; ++q) {
        const float2 dx = __fadd2_rn(f2(vel[2 * q][0], vel[2 * q + 1][0]), f2(-Un[0], -Un[0]));
        const float2 ea = __fmul2_rn(__ffma2_rn(dx, dx, f2(r2, r2)), f2(l2, l2));
        const float2 bM = __fmul2_rn(f2(pref, pref), f2(exp2_approx(ea.x), exp2_approx(ea.y)));
        const float2 o0 = __ffma2_rn(f2(ca, ca), f2(ft[0][2 * q], ft[0][2 * q + 1]), bM);
        out[0][2 * q] = o0.x; out[0][2 * q + 1] = o0.y;
        if (NC == 2) {
          const float2 o1 = __ffma2_rn(f2(ca, ca), f2(ft[NC - 1][2 * q], ft[NC - 1][2 * q + 1]),
                                       __fmul2_rn(f2(Tn, Tn), bM));
          out[NC - 1][2 * q] = o1.x; out[NC - 1][2 * q + 1] = o1.y;
        }
      }
      if (!kin[VPL - 1]) {
#pragma unroll
        for (int e = 0; e < VPL; ++e)
#pragma unroll
          for (int c = 0; c < NC; ++c) out[c][e] = kin[e] ? out[c][e] : 0.0f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VPL; ++e) {
        float c2 = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const float d = vel[e][a] - Un[a];
          c2 = fmaf(d, d, c2);
        }
        const float bM = kin[e] ? pref * __expf(nl2 * c2) : 0.0f;  // dt/(tau+dt) * M(v)
        out[0][e] = kin[e] ? fmaf(ca, ft[0][e], bM) : 0.0f;
        if (NC == 2) out[NC - 1][e] = kin[e] ? fmaf(ca, ft[NC - 1][e], Tn * bM) : 0.0f;
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) stv<S, VPL>(fo + (int64_t)c * NVp + k0, out[c]);
  }
}

// Moments of f~_i (warp totals of the lanes' compensated sums, combined in FP64; every
// lane gets them) and the relaxation of the output row.
template <typename S, int DIM, bool ROW, int VPL, int RK = 0>
__device__ __forceinline__ void finish_point(const CaseView& cv, const int i, const float* s_v,
                                             const float (&msum)[DIM + 2], const float (&mcmp)[DIM + 2]) {
  double tot[DIM + 2];
  warp_total_f64<DIM + 2>(msum, mcmp, tot);
  relax_point<S, DIM, ROW, VPL, false, RK>(cv, i, s_v, tot);
}

// Sharded step: the raw moment sums of f~_i over the slab (warp totals of the lanes'
// compensated sums, combined in FP64) to row i of the exchange buffer.
template <int DIM>
__device__ __forceinline__ void partial_out(const CaseView& cv, const int i, const float (&msum)[DIM + 2],
                                            const float (&mcmp)[DIM + 2]) {
  double tot[DIM + 2];
  warp_total_f64<DIM + 2>(msum, mcmp, tot);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) cv.xs[(int64_t)i * (DIM + 2) + q] = tot[q];
  }
}

// The per-point body, shared by the single-case kernel and the batched kernel:
// one warp, point i of case cv; s_v, s_col, s_P, s_k are this warp's shared buffers
// (nv, cap, cap * dim^2 and kahan_floats(DIM) entries).  Each lane owns VPL
// consecutive velocities of every (32 VPL)-velocity slice.  With KS the lanes'
// compensated moment sums live in s_k between slices and the velocities are
// recomputed after the neighbour loop, which keeps the 4-velocity body within 64
// registers (32 warps per SM: 0.432 against 0.465 ms with 24 on the 201^2 x 32^2 ALE
// cavity); without KS they stay in registers (the 8-velocity 3D
// body and the batched kernel, which lose with KS).  SH (sharded step): the row holds
// the velocity slab that starts at cv.vk0, and the slab's moment sums of f~ go to the
// exchange buffer instead of the relaxation.  AVG (second stage of the second-order
// step): f~ is averaged with the row of cv.f_avg and relaxed exactly over dt/2.
// KS layout: the lane's running sums and their compensations as float2 pairs, pair p of
// the sums at s_k[p * 64 + 2 lane] and of the compensations at s_k[(KP + p) * 64 + 2 lane],
// KP = (DIM + 3) / 2 (the second half of the last pair unused when DIM + 2 is odd); s_k
// is 8-byte aligned.
template <int DIM>
__host__ __device__ constexpr int kahan_pairs() { return (DIM + 3) / 2; }
template <int DIM>
__host__ __device__ constexpr int kahan_floats() { return 2 * kahan_pairs<DIM>() * 64; }

template <int DIM>
__device__ __forceinline__ void ks_store(float* s_k, const int lane, const float (&msum)[DIM + 2],
                                         const float (&mcmp)[DIM + 2]) {
  constexpr int KP = kahan_pairs<DIM>();
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const int q1 = 2 * p + 1 < DIM + 2 ? 2 * p + 1 : 2 * p;
    *reinterpret_cast<float2*>(s_k + p * 64 + 2 * lane) = f2(msum[2 * p], msum[q1]);
    *reinterpret_cast<float2*>(s_k + (KP + p) * 64 + 2 * lane) = f2(mcmp[2 * p], mcmp[q1]);
  }
}
template <int DIM>
__device__ __forceinline__ void ks_load(const float* s_k, const int lane, float (&msum)[DIM + 2],
                                        float (&mcmp)[DIM + 2]) {
  constexpr int KP = kahan_pairs<DIM>();
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const float2 a = *reinterpret_cast<const float2*>(s_k + p * 64 + 2 * lane);
    const float2 b = *reinterpret_cast<const float2*>(s_k + (KP + p) * 64 + 2 * lane);
    msum[2 * p] = a.x; mcmp[2 * p] = b.x;
    if (2 * p + 1 < DIM + 2) { msum[2 * p + 1] = a.y; mcmp[2 * p + 1] = b.y; }
  }
}

template <typename S, int DIM, bool ALE, bool ROW, int VPL, bool KS, bool SH = false, bool AVG = false>
__device__ __forceinline__ void transport_point_wp(const CaseView& cv, const int i, float* s_v, int32_t* s_col,
                                                   float* s_P, float* s_k) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  constexpr int NP = VPL / 2;  // velocity pairs per lane
  const int lane = threadIdx.x & 31;
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const int vk0 = SH ? cv.vk0 : 0;
  const float inv_nv = 1.0f / (float)nv;
  const int m = checked_count(cv.cnt[i], cap, cv.status);
  for (int q = lane; q < nv; q += 32) s_v[q] = cv.vnodes_f[q];
  {
    const int32_t* col = cv.col + (int64_t)i * cap;
    const float* P = reinterpret_cast<const float*>(cv.P) + (int64_t)i * cap * DD;
    for (int q = lane; q < m; q += 32) s_col[q] = checked_index(col[q], cv.n, i, cv.status);
    for (int q = lane; q < m * DD; q += 32) s_P[q] = P[q];
  }
  __syncwarp();

  float U[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) U[a] = ALE ? (float)cv.mom[(int64_t)i * MOM_STRIDE + 1 + a] : 0.0f;

  const int nchunk = NVp / VPL;
  const int nslice = (nchunk + 31) >> 5;
  const int64_t rowlen = (int64_t)NC * NVp;
  const S* fbase = reinterpret_cast<const S*>(cv.f_in);
  const float two_dt = cv.two_dt_f;

  // KS: s_k holds the running sums and their compensations between slices (ks_store /
  // ks_load); otherwise rsum / rcmp do
  float rsum[DIM + 2], rcmp[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) { rsum[q] = 0.0f; rcmp[q] = 0.0f; }
  if (KS) ks_store<DIM>(s_k, lane, rsum, rcmp);

  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = VPL * chunk;
    float acc[NC][VPL], sk[VPL];
    float vel[VPL][DIM];
    bool kin[VPL];
    chunk_velocities<DIM, VPL, ROW>(k0 + vk0, nv, NV + vk0, inv_nv, s_v, vel, kin);
    {
    const S* fj0 = fbase + k0;
    if (ROW) {
      // velocity pairs in packed FP32x2 arithmetic; the pairs share (v_y, v_z)
      float2 cx[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) cx[q] = f2(vel[2 * q][0] - U[0], vel[2 * q + 1][0] - U[0]);
      float crest[DIM - 1];
#pragma unroll
      for (int a = 1; a < DIM; ++a) crest[a - 1] = vel[0][a] - U[a];
      float2 skp[NP], ap[NC][NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        skp[q] = f2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < NC; ++c) ap[c][q] = f2(0.0f, 0.0f);
      }
#pragma unroll kNbrUnroll
      for (int s = 0; s < m; ++s) {
        const int j = s_col[s];
        float P[DD];
#pragma unroll
        for (int q = 0; q < DD; ++q) P[q] = s_P[s * DD + q];
        const S* fj = fj0 + (int64_t)j * rowlen;
        float fv[NC][VPL];
#pragma unroll
        for (int c = 0; c < NC; ++c) ldv_ro<S, VPL>(fj + (int64_t)c * NVp, fv[c]);
        row_upwind<DIM, NC, NP>(cx, crest, P, fv, skp, ap);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        sk[2 * q] = skp[q].x; sk[2 * q + 1] = skp[q].y;
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[c][2 * q] = ap[c][q].x; acc[c][2 * q + 1] = ap[c][q].y; }
      }
    } else {
      // velocity pairs in packed FP32x2 arithmetic; the lane's velocities need not share
      // a grid row, so each pair carries its own (c_y, c_z) and the base of c.P_d is a
      // packed product too
      float2 cx[NP], cy[NP], cz[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        cx[q] = f2(vel[2 * q][0] - U[0], vel[2 * q + 1][0] - U[0]);
        cy[q] = f2(vel[2 * q][1] - U[1], vel[2 * q + 1][1] - U[1]);
        cz[q] = DIM == 3 ? f2(vel[2 * q][DIM - 1] - U[DIM - 1], vel[2 * q + 1][DIM - 1] - U[DIM - 1]) : f2(0.0f, 0.0f);
      }
      float2 skp[NP], ap[NC][NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        skp[q] = f2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < NC; ++c) ap[c][q] = f2(0.0f, 0.0f);
      }
#pragma unroll kNbrUnroll
      for (int s = 0; s < m; ++s) {
        const int j = s_col[s];
        float P[DD];
#pragma unroll
        for (int q = 0; q < DD; ++q) P[q] = s_P[s * DD + q];
        const S* fj = fj0 + (int64_t)j * rowlen;
        float fv[NC][VPL];
#pragma unroll
        for (int c = 0; c < NC; ++c) ldv_ro<S, VPL>(fj + (int64_t)c * NVp, fv[c]);
        float2 mk[NP];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float2 px = f2(P[d * DIM], P[d * DIM]), py = f2(P[d * DIM + 1], P[d * DIM + 1]);
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            float2 bb = __fmul2_rn(cy[q], py);
            if (DIM == 3) bb = __ffma2_rn(cz[q], f2(P[d * DIM + DIM - 1], P[d * DIM + DIM - 1]), bb);
            const float2 mq = min0(__ffma2_rn(cx[q], px, bb));
            mk[q] = d == 0 ? mq : __fadd2_rn(mk[q], mq);
          }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          skp[q] = __fadd2_rn(skp[q], mk[q]);
#pragma unroll
          for (int c = 0; c < NC; ++c) ap[c][q] = __ffma2_rn(mk[q], f2(fv[c][2 * q], fv[c][2 * q + 1]), ap[c][q]);
        }
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        sk[2 * q] = skp[q].x; sk[2 * q + 1] = skp[q].y;
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[c][2 * q] = ap[c][q].x; acc[c][2 * q + 1] = ap[c][q].y; }
      }
    }
    }
    if (KS) {
      // the velocities again (not held in registers across the neighbour loop)
      chunk_velocities<DIM, VPL, ROW>(k0 + vk0, nv, NV + vk0, inv_nv, s_v, vel, kin);
      ks_load<DIM>(s_k, lane, rsum, rcmp);
    }
    slice_out<S, DIM, NC, VPL, AVG, ROW>(cv, i, k0, vel, kin, acc, sk, two_dt, rsum, rcmp);
    if (KS) {
      ks_store<DIM>(s_k, lane, rsum, rcmp);
    }
  }
  if (KS) {
    ks_load<DIM>(s_k, lane, rsum, rcmp);
  }
  if constexpr (SH) partial_out<DIM>(cv, i, rsum, rcmp);
  else finish_point<S, DIM, ROW, VPL, AVG ? 1 : 0>(cv, i, s_v, rsum, rcmp);
}

// Fixed points (the transport uses c = v): a velocity v and its mirror -v, which the
// symmetric grid stores at NV - 1 - k, share their projections p_d = v.P_d, since
//   m(v) = sum_d min(p_d, 0)  and  m(-v) = sum_d min(-p_d, 0) = m(v) - sum_d p_d.
// A lane takes the 4 consecutive velocities k0..k0+3 of a grid row in the first half
// (k0 < NV/2) and the mirror chunk NV-4-k0..NV-1-k0, whose element e holds -v_{3-e};
// so m(-v) of the lane's pair (v_{2q}, v_{2q+1}) is the mirror chunk's pair 1 - q with
// its halves swapped.  Each neighbour row then costs the projections once for 8
// velocities.  Requires nv % 4 == 0 and NV % 8 == 0 (then NVp = NV).
template <typename S, int DIM, bool KS>
__device__ __forceinline__ void transport_point_mirror(const CaseView& cv, const int i, float* s_v, int32_t* s_col,
                                                       float* s_P, float* s_k) {
  constexpr int NC = DIM == 2 ? 2 : 1;
  constexpr int DD = DIM * DIM;
  constexpr int VPL = 4, NP = 2;
  const int lane = threadIdx.x & 31;
  const int cap = cv.cap, nv = cv.nv, NV = cv.NV, NVp = cv.NVp;
  const float inv_nv = 1.0f / (float)nv;
  const int m = checked_count(cv.cnt[i], cap, cv.status);
  for (int q = lane; q < nv; q += 32) s_v[q] = cv.vnodes_f[q];
  {
    const int32_t* col = cv.col + (int64_t)i * cap;
    const float* P = reinterpret_cast<const float*>(cv.P) + (int64_t)i * cap * DD;
    for (int q = lane; q < m; q += 32) s_col[q] = checked_index(col[q], cv.n, i, cv.status);
    for (int q = lane; q < m * DD; q += 32) s_P[q] = P[q];
  }
  __syncwarp();

  const int nchunk = NV / (2 * VPL);
  const int nslice = (nchunk + 31) >> 5;
  const int64_t rowlen = (int64_t)NC * NVp;
  const S* fbase = reinterpret_cast<const S*>(cv.f_in);
  const float two_dt = cv.two_dt_f;
  const float2 neg1 = f2(-1.0f, -1.0f);

  float rsum[DIM + 2], rcmp[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) { rsum[q] = 0.0f; rcmp[q] = 0.0f; }
  if (KS) ks_store<DIM>(s_k, lane, rsum, rcmp);

  for (int sl = 0; sl < nslice; ++sl) {
    const int chunk = sl * 32 + lane;
    if (chunk >= nchunk) break;
    const int k0 = VPL * chunk, km = NV - VPL - k0;
    float acc[NC][VPL], sk[VPL], accm[NC][VPL], skm[VPL];
    {
      float vel[VPL][DIM];
      bool kin[VPL];
      chunk_velocities<DIM, VPL, true>(k0, nv, NV, inv_nv, s_v, vel, kin);
      float2 cx[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) cx[q] = f2(vel[2 * q][0], vel[2 * q + 1][0]);
      float crest[DIM - 1];
#pragma unroll
      for (int a = 1; a < DIM; ++a) crest[a - 1] = vel[0][a];
      float2 skp[NP], ap[NC][NP], skq[NP], aq[NC][NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        skp[q] = f2(0.0f, 0.0f);
        skq[q] = f2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < NC; ++c) { ap[c][q] = f2(0.0f, 0.0f); aq[c][q] = f2(0.0f, 0.0f); }
      }
      const S* fj0 = fbase + k0;
      const S* fm0 = fbase + km;
#pragma unroll 2
      for (int s = 0; s < m; ++s) {
        const int j = s_col[s];
        float P[DD];
#pragma unroll
        for (int q = 0; q < DD; ++q) P[q] = s_P[s * DD + q];
        const int64_t o = (int64_t)j * rowlen;
        float fv[NC][VPL], fw[NC][VPL];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          ldv_ro<S, VPL>(fj0 + o + (int64_t)c * NVp, fv[c]);
          ldv_ro<S, VPL>(fm0 + o + (int64_t)c * NVp, fw[c]);
        }
        float2 mk[NP], ps[NP];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          float b = crest[0] * P[d * DIM + 1];
#pragma unroll
          for (int a = 2; a < DIM; ++a) b = fmaf(crest[a - 1], P[d * DIM + a], b);
          const float2 px = f2(P[d * DIM], P[d * DIM]), bb = f2(b, b);
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const float2 p = __ffma2_rn(cx[q], px, bb);
            mk[q] = d == 0 ? min0(p) : __fadd2_rn(mk[q], min0(p));
            ps[q] = d == 0 ? p : __fadd2_rn(ps[q], p);
          }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          skp[q] = __fadd2_rn(skp[q], mk[q]);
#pragma unroll
          for (int c = 0; c < NC; ++c)
            ap[c][q] = __ffma2_rn(mk[q], f2(fv[c][2 * q], fv[c][2 * q + 1]), ap[c][q]);
          const float2 mm = __ffma2_rn(ps[q], neg1, mk[q]);  // m of (-v_{2q}, -v_{2q+1})
          const float2 mr = f2(mm.y, mm.x);                  // as mirror pair 1 - q
          const int r = NP - 1 - q;
          skq[r] = __fadd2_rn(skq[r], mr);
#pragma unroll
          for (int c = 0; c < NC; ++c)
            aq[c][r] = __ffma2_rn(mr, f2(fw[c][2 * r], fw[c][2 * r + 1]), aq[c][r]);
        }
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        sk[2 * q] = skp[q].x; sk[2 * q + 1] = skp[q].y;
        skm[2 * q] = skq[q].x; skm[2 * q + 1] = skq[q].y;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          acc[c][2 * q] = ap[c][q].x; acc[c][2 * q + 1] = ap[c][q].y;
          accm[c][2 * q] = aq[c][q].x; accm[c][2 * q + 1] = aq[c][q].y;
        }
      }
    }
    float vel[VPL][DIM], velm[VPL][DIM];
    bool kin[VPL];
    chunk_velocities<DIM, VPL, true>(k0, nv, NV, inv_nv, s_v, vel, kin);
#pragma unroll
    for (int e = 0; e < VPL; ++e)
#pragma unroll
      for (int a = 0; a < DIM; ++a) velm[e][a] = -vel[VPL - 1 - e][a];
    if (KS) {
      ks_load<DIM>(s_k, lane, rsum, rcmp);
    }
    slice_out<S, DIM, NC, VPL, false, true>(cv, i, k0, vel, kin, acc, sk, two_dt, rsum, rcmp);
    slice_out<S, DIM, NC, VPL, false, true>(cv, i, km, velm, kin, accm, skm, two_dt, rsum, rcmp);
    if (KS) {
      ks_store<DIM>(s_k, lane, rsum, rcmp);
    }
  }
  if (KS) {
    ks_load<DIM>(s_k, lane, rsum, rcmp);
  }
  finish_point<S, DIM, true, VPL>(cv, i, s_v, rsum, rcmp);
}

}  // namespace bgk
