// The ALE side chain of one step as one cooperative kernel (FP32/BF16 storage,
// skin lists): point motion (Eqs. originalALE1, ALE1), the decision to rebuild the
// candidate lists, the cell-list candidate build when it is due (Sec. 3.5.1,
// Sec. 4.2), the exact filter of the candidates, and the interior WLS stencils of
// the new lists (Sec. 3.4).  Separate launches of these steps cost a launch gap
// each on the critical path between two transports, and in most steps four of
// them would do nothing; here the phases are separated by grid-wide barriers and a
// step without a rebuild runs two phases.
//
// Every phase computes exactly what the separate kernels compute (the same device
// functions), so lists and stencils are bit-identical to them.  All blocks are
// co-resident (cooperative launch, grid from the occupancy calculator) and every
// thread reaches every barrier: the only branch around barriers is the rebuild
// decision, which every thread takes the same way.  The grid barrier is a counter
// and a generation in the case's skin state; its wait is bounded (about a second by
// default), after which the CTA records ST_TIMEOUT and returns, so the kernel cannot
// hang and no phase runs on the incomplete results of the one before it (a CTA that
// passes a barrier does so only after every CTA has arrived there).
#include <cmath>

#include "bgk_internal.cuh"
#include "device_common.cuh"
#include "motion.cuh"
#include "nbr_device.cuh"

namespace bgk {

namespace {

constexpr long long BARRIER_SPIN_LIMIT = 20000000;  // x 64 ns sleep: about a second

// Grid-wide barrier over the co-resident CTAs: the last CTA to arrive resets the
// counter and advances the generation; the others wait, at most max_spins polls, for
// the new one.  Returns false (in every thread of the CTA) when the wait gave up.
// With body non-null the last CTA to arrive also stores the body's new centre cn: it
// never waits, so the centre advances exactly once even when other CTAs give up.
__device__ __forceinline__ bool grid_barrier(SkinState* sk, DevStatus* status, long long max_spins,
                                             BodyState* body = nullptr, const double* cn = nullptr, int dim = 0) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile uint32_t* vgen = &sk->gen;
    const uint32_t g = *vgen;
    __threadfence();
    if (atomicAdd(&sk->blocks, 1u) == gridDim.x - 1) {
      // every CTA has arrived, so every thread has read the old centre
      if (body)
        for (int a = 0; a < dim; ++a) body->c[a] = cn[a];
      sk->blocks = 0u;
      __threadfence();
      atomicAdd(&sk->gen, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (++it > max_spins) {
          set_status(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int CHAIN_THREADS = 256, CHAIN_WARPS = CHAIN_THREADS / 32;
constexpr int TILE = 8;  // points per warp in the filter + stencil phase (8 groups of 4 lanes)

template <int DIM>
__global__ void __launch_bounds__(CHAIN_THREADS) k_chain(CaseView cv, double thr2, float clo, float chi, float lo,
                                                         float hi, long long max_spins) {
  extern __shared__ int32_t s_buf[];  // [CHAIN_WARPS][ccap] candidate rows
  __shared__ uint32_t s_max[CHAIN_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nthreads = (int64_t)gridDim.x * CHAIN_THREADS;
  const int64_t gtid = (int64_t)blockIdx.x * CHAIN_THREADS + threadIdx.x;
  const int gwarp = blockIdx.x * CHAIN_WARPS + warp, nwarps = gridDim.x * CHAIN_WARPS;
  SkinState* sk = cv.sk;
  const int forced = *reinterpret_cast<volatile int32_t*>(&sk->rebuild);

  // motion; the largest squared displacement since the candidate build
  double cn[3];
  body_centre_next(cv, cn);
  uint32_t dmax = 0;
  const int64_t nmov = (int64_t)cv.n_int + (cv.body ? cv.n_wall : 0);
  for (int64_t t = gtid; t < nmov; t += nthreads)
    dmax = max(dmax, __float_as_uint(__double2float_ru(move_thread(cv, (int)t, cn))));
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  if (lane == 0) s_max[warp] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0;
    for (int k = 0; k < CHAIN_WARPS; ++k) b = max(b, s_max[k]);
    atomicMax(&sk->disp2, b);
  }
  if (!grid_barrier(sk, cv.status, max_spins, cv.body, cn, cv.dim)) return;
  const uint32_t d = *reinterpret_cast<volatile uint32_t*>(&sk->disp2);
  const bool rebuild = forced || (double)__uint_as_float(d) > thr2;

  if (rebuild) {
    for (int64_t i = gtid; i < cv.n; i += nthreads) cell_assign_point(cv, (int)i);
    if (!grid_barrier(sk, cv.status, max_spins)) return;
    if (blockIdx.x == 0) {
      cell_scan_block(cv);
      // every thread has read disp2 and the rebuild flag
      if (threadIdx.x == 0) {
        sk->disp2 = 0u;
        sk->rebuild = 0;
      }
    }
    if (!grid_barrier(sk, cv.status, max_spins)) return;
    for (int64_t i = gtid; i < cv.n; i += nthreads) cell_fill_point(cv, (int)i);
    if (!grid_barrier(sk, cv.status, max_spins)) return;
    for (int i = gwarp; i < cv.n; i += nwarps)
      nbr_warp_point<DIM, true>(cv, i, lane, s_buf + warp * cv.ccap, clo, chi);
    if (!grid_barrier(sk, cv.status, max_spins)) return;
  }

  // exact lists of the new positions and the interior stencils, a tile of TILE
  // points per warp: group g = lane / 4 filters point TILE t + g and, if interior,
  // computes its stencil as k_stencils_grp does
  for (int t = gwarp; (int64_t)t * TILE < cv.n; t += nwarps) {
    const int i = t * TILE + (lane >> 2);
    const bool in = i < cv.n;
    filter_group_point<DIM>(cv, in ? i : 0, in, lane, lo, hi);
    __syncwarp();
    const bool valid = in && cv.kind[i] == 0;
    stencil_grp_point<DIM, 4>(cv, valid ? i : 0, valid, lane & 3);
  }
}

// FP32 prefilter bounds for radius r (as the separate kernels use them).
void bounds(int dim, double r, float* lo, float* hi) {
  const double r2 = r * r;
  const double band = 8.0 * dim * std::ldexp(1.0, -22) / r + std::ldexp(1.0, -16);
  *lo = band < 1.0 ? (float)(r2 * (1.0 - band)) : -1.0f;
  *hi = (float)(r2 * (1.0 + band));
}

}  // namespace

bool chain_eligible(const CaseView& cv) { return cv.ale && cv.sk && cv.storage != 0 && cv.wls_order != 2; }

// CTAs per SM of the cooperative launch (0: as many as fit, 5 at 48 registers).  The
// kernel runs beside the wall kernel; with fewer CTAs the two share the SMs instead of
// running one after the other.  201^2 x 32^2 ALE workload, ms per step (two runs each):
// all that fit 0.4932, 4 per SM 0.4929, 3 per SM 0.4900, 2 per SM 0.4895.
#ifndef BGK_CHAIN_PER_SM
#define BGK_CHAIN_PER_SM 2
#endif

int launch_chain(const CaseView& cv, int* grid_cache, long long max_spins, cudaStream_t s) {
  const size_t smem = sizeof(int32_t) * (size_t)cv.ccap * CHAIN_WARPS;
  const void* fn = cv.dim == 2 ? (const void*)k_chain<2> : (const void*)k_chain<3>;
  if (*grid_cache <= 0) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    int dev = 0, nsm = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, CHAIN_THREADS, smem) != cudaSuccess || per_sm < 1)
      return -1;
    if (BGK_CHAIN_PER_SM > 0 && per_sm > BGK_CHAIN_PER_SM) per_sm = BGK_CHAIN_PER_SM;
    *grid_cache = nsm * per_sm;
  }
  const double half = 0.5 * cv.h * cv.skin;
  double thr2 = half * half * (1.0 - 1e-6);
  float clo, chi, lo, hi;
  bounds(cv.dim, cv.h * (1.0 + cv.skin), &clo, &chi);
  bounds(cv.dim, cv.h, &lo, &hi);
  CaseView v = cv;
  long long spins = max_spins > 0 ? max_spins : BARRIER_SPIN_LIMIT;
  void* args[] = {&v, &thr2, &clo, &chi, &lo, &hi, &spins};
  if (cudaLaunchCooperativeKernel(fn, dim3(*grid_cache), dim3(CHAIN_THREADS), args, smem, s) != cudaSuccess)
    return -1;
  return 1;
}

}  // namespace bgk
