// Warp-per-point transport with the neighbour rows staged in shared memory by bulk
// copies (Sec. 3.2 transport, the same sums in the same order as transport_point_wp,
// so the results are bit-identical): each warp keeps a ring of D slots of G neighbour
// rows; lanes 0 .. 2G-1 issue one cp.async.bulk each (the g or h part of one row of
// the current velocity slice), completion is counted in bytes on the slot's mbarrier,
// and the warp refills a slot as soon as it has read it.  No CTA-wide barrier: the
// warps of a CTA run independently.  2D, FP32 storage, 4 velocities per lane that
// share a grid row (nv % 4 == 0).
#pragma once

#include "transport_wp.cuh"

namespace bgk {

#ifndef BGK_STAGE_G
#define BGK_STAGE_G 2
#endif
#ifndef BGK_STAGE_FENCE
#define BGK_STAGE_FENCE 1
#endif
#ifndef BGK_STAGE_D
#define BGK_STAGE_D 2
#endif
constexpr int kStageG = BGK_STAGE_G;  // neighbour rows per slot
constexpr int kStageD = BGK_STAGE_D;  // slots per warp
// One staged row: g and h of the 128 velocities of a slice, FP32.
constexpr int kStageRowBytes = 2 * 128 * 4;
// try_wait polls before a slot counts as lost (each poll may suspend the warp for a while).
constexpr int kStageSpins = 1 << 20;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned),
// counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits (all lanes) for the phase of `bar` with the given parity; false when it did not
// complete within kStageSpins polls (the answer is the same on every lane).
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity) {
  bool ok = mbar_try_wait(bar, parity);
  for (int spins = 0; !__all_sync(0xffffffffu, ok); ++spins) {
    if (spins >= kStageSpins) return false;
    ok = ok || mbar_try_wait(bar, parity);
  }
  return true;
}

// Shared memory of the staged kernel with W warps: the warp-per-point buffers (`base`
// bytes), then the W rings of D x G rows, then W x D mbarriers.
__host__ __device__ inline size_t stage_ring_offset(size_t base) { return (base + 127) & ~(size_t)127; }
__host__ __device__ inline size_t stage_smem_bytes(size_t base, int W) {
  return stage_ring_offset(base) + (size_t)W * kStageD * kStageG * kStageRowBytes + (size_t)W * kStageD * 8;
}

template <bool ALE>
__device__ __forceinline__ void transport_point_stage(const CaseView& cv, const int i, float* s_v, int32_t* s_col,
                                                      float* s_P, float* s_k, float* s_ring, uint64_t* s_bar) {
  constexpr int DIM = 2, NC = 2, DD = 4, VPL = 4, NP = 2, G = kStageG, D = kStageD;
  constexpr int RING_F = kStageRowBytes / 4;  // floats per staged row
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
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < D; ++b) mbar_init(s_bar + b, 1);
    fence_mbar_init();
  }
  __syncwarp();

  float U[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) U[a] = ALE ? (float)cv.mom[(int64_t)i * MOM_STRIDE + 1 + a] : 0.0f;

  const int nchunk = NVp / VPL;
  const int nslice = (nchunk + 31) >> 5;
  const int64_t rowlen = (int64_t)NC * NVp;
  const float* fbase = reinterpret_cast<const float*>(cv.f_in);
  const float two_dt = cv.two_dt_f;
  const int ng = (m + G - 1) / G;  // groups of G rows per slice
  const int ntot = nslice * ng;

  // producer cursor: the next group to issue (slice p_sl, group p_g of it, number p_t)
  int p_sl = 0, p_g = 0, p_t = 0;
  auto issue_next = [&]() {
    if (p_t >= ntot) return;
    const int b = p_t % D;
    const int s0 = p_g * G;
    const int nrow = min(G, m - s0);
    const uint32_t bytes = (uint32_t)min(32, nchunk - p_sl * 32) * 16u;
    if (lane == 0) mbar_arrive_expect_tx(s_bar + b, (uint32_t)(nrow * NC) * bytes);
    __syncwarp();
    if (lane < nrow * NC) {
      const int r = lane >> 1, c = lane & 1;
      const int j = s_col[s0 + r];
      const float* src = fbase + (int64_t)j * rowlen + (int64_t)c * NVp + p_sl * 128;
      float* dst = s_ring + (b * G + r) * RING_F + c * 128;
#if BGK_STAGE_FENCE
      fence_proxy_async();  // this warp's reads of the slot come before the copy's writes
#endif
      bulk_load(dst, src, bytes, s_bar + b);
    }
    if (++p_g == ng) { p_g = 0; ++p_sl; }
    ++p_t;
  };
#pragma unroll
  for (int q = 0; q < D; ++q) issue_next();

  float rsum[DIM + 2], rcmp[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) { rsum[q] = 0.0f; rcmp[q] = 0.0f; }
  ks_store<DIM>(s_k, lane, rsum, rcmp);

  int c_t = 0;  // consumer: the next group to read
  bool lost = false;
  for (int sl = 0; sl < nslice && !lost; ++sl) {
    const int chunk = sl * 32 + lane;
    const bool act = chunk < nchunk;  // lanes past the last chunk keep to the warp's waits only
    const int k0 = VPL * chunk;
    float acc[NC][VPL], sk[VPL];
    float vel[VPL][DIM];
    bool kin[VPL];
    chunk_velocities<DIM, VPL, true>(k0, nv, NV, inv_nv, s_v, vel, kin);
    float2 cx[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) cx[q] = f2(vel[2 * q][0] - U[0], vel[2 * q + 1][0] - U[0]);
    float crest[DIM - 1];
    crest[0] = vel[0][1] - U[1];
    float2 skp[NP], ap[NC][NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      skp[q] = f2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < NC; ++c) ap[c][q] = f2(0.0f, 0.0f);
    }
    for (int g = 0; g < ng; ++g, ++c_t) {
      const int b = c_t % D;
      if (!stage_wait(s_bar + b, (uint32_t)(c_t / D) & 1u)) { lost = true; break; }
      const int s0 = g * G;
      const float* slot = s_ring + b * G * RING_F + 4 * lane;
#pragma unroll
      for (int r = 0; r < G; ++r) {
        if (s0 + r < m) {
          const float4 p4 = reinterpret_cast<const float4*>(s_P)[s0 + r];
          const float P[DD] = {p4.x, p4.y, p4.z, p4.w};
          const float4 a = *reinterpret_cast<const float4*>(slot + r * RING_F);
          const float4 h = *reinterpret_cast<const float4*>(slot + r * RING_F + 128);
          const float fv[NC][VPL] = {{a.x, a.y, a.z, a.w}, {h.x, h.y, h.z, h.w}};
          row_upwind<DIM, NC, NP>(cx, crest, P, fv, skp, ap);
        }
      }
      __syncwarp();
      issue_next();
    }
    if (lost) break;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      sk[2 * q] = skp[q].x; sk[2 * q + 1] = skp[q].y;
#pragma unroll
      for (int c = 0; c < NC; ++c) { acc[c][2 * q] = ap[c][q].x; acc[c][2 * q + 1] = ap[c][q].y; }
    }
    if (act) {
      chunk_velocities<DIM, VPL, true>(k0, nv, NV, inv_nv, s_v, vel, kin);
      ks_load<DIM>(s_k, lane, rsum, rcmp);
      slice_out<float, DIM, NC, VPL, false, true>(cv, i, k0, vel, kin, acc, sk, two_dt, rsum, rcmp);
      ks_store<DIM>(s_k, lane, rsum, rcmp);
    }
    __syncwarp();
  }
  if (lost) {
    // a slot never completed: flag it, wait (bounded) for this warp's other copies in
    // flight so that none lands after the CTA has left, and leave the point unrelaxed
    if (lane == 0) set_status(cv.status, ST_TIMEOUT);
    for (int t = c_t + 1; t < p_t; ++t) (void)stage_wait(s_bar + t % D, (uint32_t)(t / D) & 1u);
    return;
  }
  ks_load<DIM>(s_k, lane, rsum, rcmp);
  finish_point<float, DIM, true, VPL>(cv, i, s_v, rsum, rcmp);
}

}  // namespace bgk
