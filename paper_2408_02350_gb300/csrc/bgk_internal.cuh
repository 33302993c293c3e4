// Internal declarations shared by the CUDA translation units of libbgk.
// Device data of one problem ("case") and the host-side launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace bgk {

// Device status bits (reported by bgk_sync).
enum : int32_t { ST_OVERFLOW = 1, ST_SINGULAR = 2, ST_NONFINITE = 4, ST_TIMEOUT = 8, ST_BOUNDS = 16 };

// Verlet-list state of an ALE case: the largest squared displacement of an interior
// point since the candidate build (FP32 bits, rounded up), the rebuild decision for
// the next list build (taken by the last CTA of the motion kernel or by the
// side-chain kernel; set by the host whenever positions or lists are reset), the CTA
// counter of those kernels (zero between kernels) and the generation of the
// side-chain kernel's grid barrier.
struct SkinState {
  uint32_t disp2;
  int32_t rebuild;
  uint32_t blocks;
  uint32_t gen;
};

// Rigid body (body_wall > 0): its current centre and the CTA counter of the motion
// kernel, whose last CTA advances the centre after every CTA has read it.
struct BodyState {
  double c[3];
  uint32_t blocks;
  int32_t pad;
};

struct DevStatus {
  int32_t flags;
  int32_t pad;
  unsigned long long clamps;

};

// Moments are stored per point as MOM_STRIDE doubles: rho, U[3], T.
constexpr int MOM_STRIDE = 5;

// Everything a kernel needs about one case, passed by value.  All pointers are
// device pointers owned by the context.
struct CaseView {
  int32_t dim, nv, NV, NVp, ncomp, cap;
  int32_t n, n_int, n_wall;
  int32_t ale, periodic, tau_mode, lid_wall, storage;
  int32_t nc, ncell;  // cells per axis, total cells
  double dt, h, alpha, kn, wall_T, guard, dv;
  double lid_u[3];
  // set on the host with the values above (set_case_consts): the quadrature weight dv^dim
  // and FP32 copies of per-case constants, so that the FP32 kernels convert nothing per
  // point (conversions from FP64 run on the FP64 pipe, a small fraction of the FP32 rate)
  double wv, h2;  // dv^dim; h^2 (IEEE double product, as the exact neighbour test takes it)
  float dt_f, two_dt_f, kn_f, wv_f;
  float nah2_f, inv_h_f;  // -alpha / h^2 and 1 / h in FP32 (Gaussian weights of the FP32 stencils)

  double* vnodes;          // [nv] velocity nodes (FP64)
  float* vnodes_f;         // [nv] the same nodes rounded to FP32
  double* x;               // [n][dim]
  const int32_t* kind;     // [n]
  const double* normal;    // [n][dim]
  const int32_t* int_idx;  // [n_int] interior point indices, Morton order of the initial positions
  const int32_t* wall_idx; // [n_wall] wall point indices, ascending

  float* xf;            // [n][dim] FP32 rounding of x (neighbour-search prefilter, high part)
  float* xlo;           // [n][dim] FP32 x - xf (low part): xf + xlo carries x to ~2^-48
  int32_t* cell_of;     // [n]
  int32_t* cell_start;  // [ncell + 1]
  int32_t* cell_cnt;    // [ncell]
  int32_t* cell_pts;    // [n]

  int32_t* cnt;  // [n]
  int32_t* col;  // [n][cap]
  void* P;       // [n][cap][dim*dim] projected frame vectors, compute type
  void* recon;   // [n][cap] wall reconstruction weights, compute type

  // wall tables: per wall slot w = 0..n_wall-1, with c_n = (v - u_w).n the normal
  // velocity relative to the wall (constant in time: walls at rest, the lid moving
  // tangentially, the body translating without rotation)
  int8_t* wcls;    // [n_wall][NVp] 1 leaving (c_n > 0), 0 arriving
  void* wvn;       // [n_wall][NVp] |c_n|, compute type
  double* winv;    // [n_wall] 1 / sum_{c_n>0} c_n M_w(v)
  void* mw;        // [3][NVp] wall Maxwellian G1 (or M) with rho = 1: [0] at rest, [1] lid, [2] body

  void* f_in;    // [n][ncomp][NVp] storage type
  void* f_out;   // [n][ncomp][NVp] storage type
  float* ft_out; // optional [n][ncomp][NVp] copy of the transported f~ (FP32 path, adjoint recomputation)
  float* sk_out; // optional [n][NVp] sum_j min-terms of the upwind coefficients (diagonal of the transport)
  double* mom;   // [n][MOM_STRIDE]
  DevStatus* status;

  // ALE neighbour-list skin (null / 0 when not used): candidate lists of radius h (1 + skin)
  double skin;          // fraction of h
  int32_t ccap;         // candidate-list capacity
  double* xb;           // [n][dim] positions at the last candidate build
  int32_t* ccnt;        // [n]
  int32_t* ccol;        // [n][ccap] candidates, ascending
  SkinState* sk;

  // rigid body (body_wall = 0: none)
  int32_t body_wall;
  int32_t wls_order;  // 2: second-order Taylor fit for the interior stencils, else linear
  double body_u[3];
  double body_rg;       // guard radius body_radius + guard
  BodyState* body;

  // velocity slab of a sharded case: its rows of f hold the velocities with flattened
  // grid index vk0 .. vk0 + NV - 1 (vk0 = 0 and NV = nv^dim for the whole grid)
  int32_t vk0;
  int32_t pad_vk;
  double* xs;  // exchange buffer of the current sharded phase (device, caller-owned), else null
  // second-order step: the state at the start of the step, averaged into the second
  // transport stage (null otherwise)
  void* f_avg;
};

// The derived per-case constants of CaseView (wv, h2 and the FP32 copies), from dim, dt,
// kn, dv, h, alpha.
inline void set_case_consts(CaseView& v) {
  v.wv = v.dim == 2 ? v.dv * v.dv : v.dv * v.dv * v.dv;
  v.h2 = v.h * v.h;
  v.nah2_f = (float)(-v.alpha / (v.h * v.h));
  v.inv_h_f = (float)(1.0 / v.h);
  v.dt_f = (float)v.dt;
  v.two_dt_f = (float)(2.0 * v.dt);
  v.kn_f = (float)v.kn;
  v.wv_f = (float)v.wv;
}

// Launchers (stream-ordered; each returns the number of kernels launched).
int launch_init_tables(const CaseView& cv, cudaStream_t s);
int launch_neighbours(const CaseView& cv, cudaStream_t s);
// Point management (between steps): plan (nearest pairs, roles, new indices; totals[0] =
// survivors, totals[1] = additions requested) and apply (new positions, rows of f,
// index lists) for n_new = survivors + min(additions, cap_n - survivors) points.
int launch_manage_plan(const CaseView& cv, double rmin, int min_nbrs, int32_t* nn, int32_t* role, double* ynew,
                       int32_t* newidx, int32_t* addidx, int32_t* totals, cudaStream_t s);
int launch_manage_apply(const CaseView& cv, int64_t cap_n, const int32_t* nn, const int32_t* role,
                        const double* ynew, const int32_t* newidx, const int32_t* addidx, const int32_t* totals,
                        double* x2, int32_t* kind2, double* norm2, const void* f, void* f2, int32_t* int2,
                        int32_t* wall_idx, int32_t* wall_of, int64_t n_new, cudaStream_t s);
// ALE with a skin: rebuild the candidate lists if a point moved too far, then filter them.
int launch_neighbours_skin(const CaseView& cv, cudaStream_t s);
// ALE with a skin, FP32/BF16 storage: motion, candidate rebuild when due, filter and
// interior stencils of the list set in cv as one cooperative launch (grid size cached
// in *grid_cache); returns 1, or -1 when the cooperative launch is unavailable.  A grid
// barrier waits at most max_spins polls (0: about a second), then the kernel records
// ST_TIMEOUT and its CTAs return.
bool chain_eligible(const CaseView& cv);
int launch_chain(const CaseView& cv, int* grid_cache, long long max_spins, cudaStream_t s);
// Velocity-sharded step (slabs of the velocity grid, coupled only through velocity sums;
// cv.xs is the exchange buffer of the phase):
//  transport: f~ of the slab into f_out, raw moment sums of f~ over the slab into
//             xs[i][dim + 2] (interior rows i);
//  relax:     moments of interior points from the summed xs, relaxation of f_out in place;
//  walls 1:   arriving half of every wall row and the wall sums xs[w][2 dim + 6];
//  walls 2:   leaving half and the wall moments from the summed xs;
//  partial:   raw moment sums of f_in over the slab, xs[i][dim + 2] for every point;
//  moments:   moments of every point from the summed xs;
//  allreduce: sum of nbufs device buffers of count doubles into each of them.
int launch_shard_transport(const CaseView& cv, cudaStream_t s);
int launch_shard_relax(const CaseView& cv, cudaStream_t s);
int launch_shard_walls(const CaseView& cv, int phase, cudaStream_t s);
int launch_shard_partial(const CaseView& cv, cudaStream_t s);
int launch_shard_moments(const CaseView& cv, cudaStream_t s);
int launch_shard_allreduce(double* const* bufs, int nbufs, int64_t count, cudaStream_t s);
constexpr int SHARD_MAX_BUFS = 16;
// part 0: all points; 1: interior stencils (all points for FP64 storage); 2: wall
// reconstruction weights (nothing for FP64 storage).
int launch_stencils(const CaseView& cv, cudaStream_t s, int part = 0);
int launch_transport(const CaseView& cv, cudaStream_t s);
// Second-order step (fixed points): the second transport stage, f~ averaged with the row of
// cv.f_avg and relaxed exactly over dt/2 into f_out; and the exact relaxation over dt/2 of
// f_out in place with the moments of its own rows (interior points).
int launch_transport_avg(const CaseView& cv, cudaStream_t s);
int launch_relax_half(const CaseView& cv, cudaStream_t s);
// FP32 warp-per-point transport + relaxation (used by the adjoint's forward recomputation)
int launch_transport_fp32(const CaseView& cv, cudaStream_t s);
int launch_walls(const CaseView& cv, cudaStream_t s);
// Batched (many cases, one launch each): FP32/BF16 storage, all cases of one dimension.
int launch_transport_batch(const CaseView* d_cases, const int2* items, int n_items, int dim, int storage, int capmax,
                           int warps, int grid, cudaStream_t s);
int launch_walls_batch(const CaseView* d_cases, const int2* witems, int n_witems, int dim, int storage, int capmax,
                       cudaStream_t s);
int launch_move(const CaseView& cv, cudaStream_t s);
int launch_set_maxwellian(const CaseView& cv, double rho0, const double* u0, double T0, cudaStream_t s);
int launch_moments(const CaseView& cv, const void* f, cudaStream_t s);
// Convert between a dense user layout [n][ncomp][NV] of type src_dtype and the
// internal padded storage [n][ncomp][NVp].
int launch_pack_f(const CaseView& cv, const void* src, int src_dtype, void* dst, cudaStream_t s);
int launch_unpack_f(const CaseView& cv, const void* src, void* dst, int dst_dtype, cudaStream_t s);
// Stencils of every neighbour slot in CSR order, converted to double (device
// destination arrays P[nnz][dim*dim], recon[nnz]; rowptr[n+1] on the device).
int launch_stencils_csr(const CaseView& cv, const int64_t* rowptr, double* P, double* recon, cudaStream_t s);

// Discrete adjoint (adjoint.cu): transpose slot map, one adjoint step, objective.
int launch_tslot(const CaseView& cv, int32_t* tslot, cudaStream_t s);
int launch_adjoint(const CaseView& cv, const void* lam1, void* lam0, double* dtheta, void* FT, void* Y, void* LFT,
                   double* wmu, const int32_t* tslot, const int32_t* wall_of, cudaStream_t s);
int launch_adjoint_fp32(const CaseView& cv, const void* lam1, void* lam0, double* dtheta, void* FT, void* Y, void* LFT,
                        double* wmu, double* amom, float* SK, const int32_t* tslot, const int32_t* wall_of, cudaStream_t s);
int launch_objective(const CaseView& cv, int nlid, double* J, void* lam, double scale, cudaStream_t s);

// Kernel ids for timing.
enum KernelId { K_TRANSPORT = 0, K_WALLS = 1, K_NBR = 2, K_STENCIL = 3, K_MOVE = 4, K_ADJOINT = 5, K_BATCH = 6, K_COUNT = 7 };

}  // namespace bgk
