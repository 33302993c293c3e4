/*
 * bgk.h -- C ABI of the GB300 library for one time step of the meshfree
 * Arbitrary-Lagrangian-Eulerian / weighted-least-squares scheme for the BGK
 * equation (Mariappan, Willems, Boregowda, Tiwari, Klar, arXiv 2408.02350).
 *
 * Every call takes plain pointers and sizes.  Conventions for all calls:
 *  - The return value is a bgk_status.  No call aborts, traps or prints;
 *    bgk_last_error(ctx) gives a one-line description of the last failure.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream are asynchronous with respect to the
 *    host and ordered on that stream, except where noted as synchronous.
 *  - Device-side failures (neighbour overflow, singular WLS system,
 *    non-finite moments) are recorded in a device status word and returned by
 *    the next bgk_sync.
 *  - The caller owns every pointer it passes.  The context owns all device
 *    memory it allocates (positions, neighbour lists, stencils, the two
 *    distribution buffers) and frees it in bgk_free.
 *  - Units are nondimensional: R = 1, L = 1, rho0 = 1, T0 = 1.
 *
 * Layouts:
 *   x, normal  [n][dim] double, row-major
 *   kind       [n] int32: 0 interior point, k > 0 wall id
 *   f          [n][ncomp][NV] with ncomp = 2 (Chu g1, g2) in 2D, 1 in 3D,
 *              NV = nv^dim, velocity index k = kx + nv*(ky + nv*kz)
 *   velocity nodes v_j = -vmax + j*dv, dv = 2 vmax / (nv - 1), j = 0..nv-1
 *              (vgrid = 1: v_j = -vmax + (j + 1/2) dv, dv = 2 vmax / nv)
 */
#ifndef BGK_H
#define BGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BGK_ABI_VERSION 9

typedef struct bgk_ctx bgk_ctx;

typedef enum bgk_status {
  BGK_OK = 0,
  BGK_E_INVAL = 1,         /* bad argument or size */
  BGK_E_NOMEM = 2,         /* device or host allocation failed */
  BGK_E_CUDA = 3,          /* a CUDA runtime call failed */
  BGK_E_SINGULAR = 4,      /* WLS normal matrix not invertible, or a wall point without interior neighbours */
  BGK_E_NBR_OVERFLOW = 5,  /* a point has more than max_nbrs neighbours */
  BGK_E_NONFINITE = 6,     /* non-finite or non-positive density or temperature */
  BGK_E_TIMEOUT = 7,       /* a bounded device wait gave up */
  BGK_E_STATE = 8,         /* call not valid in the context's state */
  BGK_E_BOUNDS = 9         /* (bounds-checked debug build only) a neighbour or point index
                              outside the point range was found and its access skipped */
} bgk_status;

typedef enum bgk_storage { BGK_F64 = 0, BGK_F32 = 1, BGK_BF16 = 2 } bgk_storage;

typedef enum bgk_tau_mode {
  BGK_TAU_LOCAL = 0,   /* tau = sqrt(2/pi) Kn / (rho sqrt(T)), Eqs. (tau), (lambda) */
  BGK_TAU_CONST = 1,   /* tau = sqrt(2/pi) Kn */
  BGK_TAU_NONE = 2     /* no collisions (free transport) */
} bgk_tau_mode;

/* Parameters of one problem (Sec. 3 and Sec. 5). */
typedef struct bgk_params {
  int32_t dim;       /* 2: Chu-reduced g1, g2 (Sec. 2.1); 3: full f */
  int32_t nv;        /* velocity nodes per axis (the paper's N_v + 1), >= 2 */
  double vmax;       /* velocity grid covers [-vmax, vmax]^dim (Sec. 3.3) */
  double kn;         /* Knudsen number */
  int32_t tau_mode;  /* bgk_tau_mode */
  int32_t ale;       /* 1: points move with U and transport uses v - U (Sec. 3.1) */
  int32_t periodic;  /* 1: periodic unit box (minimum image), no walls */
  int32_t lid_wall;  /* wall id whose points move with lid_u (diffuse reflection) */
  int32_t max_nbrs;  /* neighbour-list capacity per point */
  int32_t storage;   /* bgk_storage of f: F64 computes in double, F32/BF16 in float,
                        except that the WLS normal matrices are accumulated and solved
                        and the moment sums combined (rho, U, T formed) in double for
                        every storage type */
  double dt;         /* time step */
  double h;          /* neighbour radius and WLS support (Sec. 3.4.1) */
  double alpha;      /* Gaussian weight w = exp(-alpha r^2 / h^2), Eq. (weight) */
  double wall_T;     /* wall temperature */
  double guard;      /* ALE: interior coordinates are clamped to [guard, 1 - guard] */
  double lid_u[3];   /* lid velocity */
  double skin;       /* ALE neighbour-list skin, a fraction of h in [0, 1]: candidate
                        lists of radius h (1 + skin) are built with the cell search and
                        re-filtered with the exact test every step, and rebuilt once a
                        point has moved more than h skin / 2 since the last build.  The
                        lists equal those of a full search every step; 0 turns it off.
                        Fixed at bgk_init. */
  int32_t spare_points; /* room for points that bgk_manage may add beyond the initial
                           count (every per-point array holds n + spare_points) */
  int32_t pad2_;
  /* Rigid body moving through the gas (Sec. 3.4.1: boundary points move together
   * with a moving boundary).  body_wall > 0 is the wall id of the body's boundary
   * points (not lid_wall); 0 means no body.  Each step (ale = 1) the body's centre
   * and boundary points advance by dt body_u, computed as x + dt*u in FP64 without
   * fused multiply-add; body_u is also their wall velocity, so the diffuse reflection
   * classifies velocities by (v - body_u).n and emits M(v; rho_w, body_u, wall_T).
   * Interior points that end a step closer than body_radius + guard to the centre
   * are put back on that sphere along the ray from the centre (counted as clamps),
   * and bgk_manage adds no point inside it.  body_wall, body_centre and
   * body_radius are fixed at bgk_init; body_u may change through bgk_set_params
   * and must be zero unless ale = 1.  (wls_order, between body_wall and body_u, is
   * described at its field.) */
  int32_t body_wall;
  int32_t wls_order;     /* interior derivative stencils from the linear (0 or 1: the paper's
                            scheme) or the second-order (2) Taylor expansion of Sec. 3.4.1;
                            the second-order fit needs dim + dim (dim + 1) / 2 neighbours per
                            point and is solved in FP64 for every storage type.  Fixed at
                            bgk_init. */
  double body_u[3];      /* body velocity */
  double body_centre[3]; /* centre of the body at bgk_init */
  double body_radius;    /* radius of the body's guard sphere (without guard) */
  /* Velocity slab for the sharded step (bgk_shard_*): the case holds only the
   * velocities with flattened grid index k in [vk_lo, vk_hi), and every layout of f
   * ([n][ncomp][NV]) then has NV = vk_hi - vk_lo.  vk_hi = 0 (with vk_lo = 0) holds
   * the whole grid.  vk_lo must be a multiple of 4.  Fixed at bgk_init. */
  int32_t vk_lo;
  int32_t vk_hi;
  /* Time discretisation.  0 or 1: the paper's first-order splitting (Sec. 3.2: explicit
   * upwind transport, implicit relaxation).  2: a second-order variant, which the paper
   * leaves to future work (Sec. 6): Strang splitting f^{n+1} = R(dt/2) T(dt) R(dt/2) f^n
   * with the relaxation solved exactly (it keeps rho, U and T, so R(h) f = M + (f - M)
   * exp(-h / tau)) and T two explicit transport stages (Heun):
   * f^T = (f + T1(T1 f)) / 2 with T1 the first-order transport and the walls applied to
   * each stage.  Needs ale = 0; not with bgk_shard_*, the batched modes or the adjoint.
   * Fixed at bgk_init. */
  int32_t time_order;
  /* Velocity grid (Sec. 3.3): 0 the paper's nv nodes from -vmax to vmax, dv = 2 vmax /
   * (nv - 1); 1 the midpoint grid, nv cells of width dv = 2 vmax / nv with a node at each
   * cell centre (no node at +-vmax).  Both are symmetric about zero.  Fixed at bgk_init. */
  int32_t vgrid;
} bgk_params;

typedef struct bgk_stats {
  int64_t steps;          /* time steps taken */
  int64_t launches;       /* kernels launched by this context since creation */
  int64_t clamps;         /* ALE wall-guard clamps (valid after bgk_sync) */
  int64_t nnz;            /* neighbour pairs in the current lists, all cases */
  int32_t nv_pad;         /* padded velocity stride of the internal f layout */
  int32_t n_cases;
  int32_t batch_mode;     /* stepping mode in effect: 0 per case, 1 batched kernels, 2 batched kernels in a graph */
  int32_t batch_warps;    /* warps per CTA of the batched transport (bgk_autotune) */
  int32_t batch_grid;     /* CTAs of the persistent batched transport, 0 = one per tile (bgk_autotune) */
  int32_t pad_;
} bgk_stats;

/* Library ABI version (BGK_ABI_VERSION). */
int bgk_version(void);

/* Failure detection (not in the paper): the number of polls after which a bounded
 * device wait gives up (the grid barriers of the fused ALE list-build kernel); 0
 * restores the default of about one second.  A wait that gives up records
 * BGK_E_TIMEOUT for the next bgk_sync and its CTAs leave the kernel, so no later phase
 * runs on incomplete data.  The motion before the first wait is complete; the lists
 * of the new positions are partly stale (every index still valid), and a step taken
 * before the bgk_sync that reports the timeout runs on them.  That bgk_sync resets the
 * waits' state and discards those lists, so the step after it builds its lists from
 * the positions and the run continues as one without a timeout.  A limit of 1 makes
 * the waits give up at once, which tests that path without a hang. */
int bgk_set_watchdog(bgk_ctx* ctx, int64_t max_polls);

/* Measurement support, not part of the method: the FP32 fused-multiply-add rate of
 * the current device (the ceiling of the ALU-bound transport), from a kernel in which
 * every thread runs 8 independent FMA chains on 8 CTAs of 256 threads per SM, timed
 * with CUDA events (best of three after a warm-up launch).  fma_per_s: scalar FMAs per
 * second; fma2_per_s: FMAs per second with packed pairs; n_sm: the multiprocessor
 * count.  Synchronous; a few ms. */
int bgk_peak_fp32(double* fma_per_s, double* fma2_per_s, int32_t* n_sm, void* stream);

/* The same for FP64: dfma_per_s = FP64 FMAs per second (the ceiling of the plain FP64
 * path).  Synchronous. */
int bgk_peak_fp64(double* dfma_per_s, void* stream);

/* Create a context for n_cases independent problems (Sec. 5; several cavities
 * of different sizes and parameters may share one context).  p[n_cases],
 * n_points[n_cases]; x, kind, normal are host arrays concatenated over the
 * cases.  Copies the geometry to the current CUDA device and allocates every
 * device buffer.  f is not initialised until bgk_set_maxwellian or bgk_set_f.
 * Positions lie in the unit box [0, 1]^dim (the cell grid of the neighbour search
 * spans it), kind is 0 for an interior point and a wall id > 0 otherwise, normals are
 * finite.  Synchronous.  Returns BGK_E_INVAL, before touching the device, for an
 * unsupported parameter, a non-finite or out-of-box coordinate, a negative kind or a
 * non-finite normal. */
int bgk_init(const bgk_params* p, int32_t n_cases, const int64_t* n_points, const double* x,
             const int32_t* kind, const double* normal, bgk_ctx** out);

/* f^0 = Maxwellian(rho0, u0[dim], T0) at every point of every case
 * (Sec. 2.1: g1 = G1, g2 = T0 G1 in 2D), and the stored moments (rho, U, T)
 * are those of f^0 (the transport of the first step uses their U).  A case that
 * holds a proper velocity slab (vk_lo, vk_hi) gets its slab of f^0 only; its
 * moments come from bgk_shard_partial and bgk_shard_set_moments. */
int bgk_set_maxwellian(bgk_ctx* ctx, double rho0, const double* u0, double T0, void* stream);

/* Copy case c's distribution in or out, layout [n][ncomp][NV] with element
 * type dtype (bgk_storage), from/to host memory (on_device = 0) or device
 * memory (on_device = 1).  bgk_set_f also recomputes the stored moments (not for
 * a proper velocity slab: see bgk_set_maxwellian).
 * Host copies are synchronous (direct between host memory and the distribution
 * buffer when dtype is the storage type and NV needs no padding, else staged
 * and converted on the device); device copies are stream-ordered. */
int bgk_set_f(bgk_ctx* ctx, int32_t c, const void* f, int32_t dtype, int32_t on_device, void* stream);
int bgk_get_f(bgk_ctx* ctx, int32_t c, void* f, int32_t dtype, int32_t on_device, void* stream);

/* Upload case c's distribution for the next bgk_step without waiting: f is
 * page-locked host memory, layout [n][ncomp][NV] of the storage type (NV a multiple of
 * 4).  The copy goes into a third device buffer on internal streams (four copies of
 * a quarter of the rows each, so that several copy engines share it), so it overlaps
 * whatever runs meanwhile (the step before, typically); the next bgk_step waits for it
 * on its stream, takes it as the state (as bgk_set_f would, moments included) and steps
 * from it.  A second call before that step replaces the pending input; bgk_manage and
 * bgk_set_state drop it.  f must stay unchanged until the copy has run (any call that
 * waits for the stream after the next bgk_step ensures it).  BGK_E_STATE with bound
 * storage (bgk_bind_f) or for a velocity slab; BGK_E_INVAL for pageable memory or
 * another element type.  Asynchronous. */
int bgk_stage_f(bgk_ctx* ctx, int32_t c, const void* f, int32_t dtype);

/* Caller-owned storage for case c's distribution (no copies per step): f_dev is
 * device memory of at least (n + spare_points) ncomp NV elements of the storage type,
 * 16-byte aligned, layout [n][ncomp][NV]; NV must be a multiple of 4 (then the
 * internal layout is this one).  The call copies the current state into f_dev, and
 * from then on every call leaves the case's state in f_dev when it returns: the
 * context's own second buffer still serves the double buffering, and a call that ends
 * with the state there copies it into f_dev (one device copy; bgk_step with an even
 * step count needs none).  The context never frees f_dev.  After writing into f_dev,
 * call bgk_set_f with f_dev itself (on_device = 1, the storage type) to recompute the
 * stored moments; nothing is copied then.  f_dev = NULL unbinds: the state goes back
 * into the context's own buffer, and the call waits for the stream, after which the
 * caller may free the memory.  Rebinding unbinds first.  BGK_E_INVAL for a buffer that
 * is too small, misaligned or not device memory; BGK_E_STATE while an input staged by
 * bgk_stage_f is pending.  Stream-ordered except the unbinding. */
int bgk_bind_f(bgk_ctx* ctx, int32_t c, void* f_dev, size_t bytes, void* stream);

/* Rebuild cell lists, neighbour lists N(i) = {j != i : |x_j - x_i|^2 <= h^2}
 * (ascending j, FP64 without fused multiply-add) and the WLS stencils of
 * every case from the current positions (Sec. 3.4, Sec. 3.5.1, Sec. 4.2).
 * bgk_step does this itself: every step when ale = 1, once otherwise. */
int bgk_neighbours(bgk_ctx* ctx, void* stream);

/* Host copy of case c's neighbour lists as CSR: rowptr[n+1], col[cap]: the
 * lists the last step used (after bgk_neighbours: the lists it built).
 * *nnz receives the pair count; BGK_E_INVAL if cap < nnz.  Synchronous. */
int bgk_get_neighbours(bgk_ctx* ctx, int32_t c, int64_t* rowptr, int32_t* col, int64_t cap, int64_t* nnz);

/* Host copy of case c's stencils in neighbour-list order (CSR slots):
 * P[nnz][dim][dim] holds, for interior rows, the projected frame vectors
 * abar_d e_d (d = n, t[, b]) of Sec. 3.4.2 so that the upwind coefficient is
 * K = sum_d (c.P_d - |c.P_d|); recon[nnz] holds, for wall rows, the WLS
 * reconstruction weights (zero for wall neighbours).  Synchronous. */
int bgk_get_stencils(bgk_ctx* ctx, int32_t c, double* P, double* recon, int64_t cap);

/* Advance every case by nsteps time steps of the first-order splitting of
 * Sec. 3.2: positive upwind transport f~ = f - dt (v - U^n).grad f (Sec. 3.4.2),
 * moments of f~ (Eqs. fullmoment1a, moment1a, moment1b), implicit BGK
 * relaxation f^{n+1} = (tau f~ + dt M^{n+1}) / (tau + dt), diffuse-reflection
 * walls, and with ale = 1 the motion x^{n+1} = x^n + dt U^{n+1}.  Asynchronous:
 * with ale = 1 the motion and the next step's lists run on an internal stream
 * concurrently with the wall kernel, and every such piece of work is ordered
 * before later work on `stream` when the call returns.  A case with time_order = 2
 * takes the second-order step described at that field instead.  BGK_E_STATE when a
 * case holds a proper velocity slab (such cases step with bgk_shard_*). */
int bgk_step(bgk_ctx* ctx, int32_t nsteps, void* stream);

/* Velocity-sharded step, not in the paper (Sec. 5 parallelises over points on one
 * GPU): the step split over the discrete velocities, for several GPUs.  R cases -- in R contexts on R GPUs, or in one or several contexts on one GPU --
 * hold the same points and disjoint velocity slabs [vk_lo, vk_hi) that cover the
 * grid.  Transport and relaxation act on each velocity separately; the slabs couple
 * only through sums over velocities, so positions, neighbour lists, stencils and
 * moments are replicated and evolve identically in every slab as long as each slab
 * receives the same sums.  One step of case c of every slab is
 *   bgk_shard_transport(xm)       then xm <- sum of xm over the slabs (allreduce)
 *   bgk_shard_relax(xm, xw)       then xw <- sum of xw over the slabs (allreduce)
 *   bgk_shard_walls(xw)
 * and equals a bgk_step of the whole grid up to the order of the velocity sums.
 * Exchange buffers are caller-owned device arrays of doubles:
 *   xm  [n][dim + 2]      raw moment sums (sum g, sum v g, sum |v|^2 g (+ sum h))
 *                         of f~ (transport: interior rows; other rows untouched)
 *                         or of f (bgk_shard_partial: every row)
 *   xw  [n_wall][2 dim + 6], wall points in ascending index order: sum over the
 *       arriving velocities of |c_n| g, sum over the leaving ones of c_n M_w, the
 *       moment sums of the arriving half, those of M_w over the leaving half
 * (bgk_shard_sizes gives the two lengths; xw may be NULL when the case has no wall
 * points).  The buffers must stay valid until the stream has run the call's kernels;
 * the summed buffer must hold identical bits in every slab (NCCL's allreduce and
 * bgk_shard_allreduce both do).  Calls out of this
 * order return BGK_E_STATE.  Stream-ordered.  With ale = 1 the motion and the next
 * lists run on the internal stream after bgk_shard_relax, as in bgk_step.
 * bgk_stats.steps counts the bgk_shard_walls calls of case 0. */
int bgk_shard_sizes(bgk_ctx* ctx, int32_t c, int64_t* n_xm, int64_t* n_xw);
int bgk_shard_transport(bgk_ctx* ctx, int32_t c, double* xm, void* stream);
int bgk_shard_relax(bgk_ctx* ctx, int32_t c, const double* xm, double* xw, void* stream);
int bgk_shard_walls(bgk_ctx* ctx, int32_t c, const double* xw, void* stream);

/* Stored moments of a sharded case from its current f: bgk_shard_partial writes the
 * slab's raw sums of every point to xm, and after the sum over the slabs
 * bgk_shard_set_moments sets (rho, U, T) of every point from it (after
 * bgk_set_maxwellian, bgk_set_f or bgk_set_state).  Stream-ordered. */
int bgk_shard_partial(bgk_ctx* ctx, int32_t c, double* xm, void* stream);
int bgk_shard_set_moments(bgk_ctx* ctx, int32_t c, const double* xm, void* stream);

/* Sum for slabs that share one GPU: bufs[nbufs] device arrays of count doubles
 * (1 <= nbufs <= 16); every element becomes the sum over the buffers, added in
 * buffer order, in every buffer.  Stream-ordered. */
int bgk_shard_allreduce(double* const* bufs, int32_t nbufs, int64_t count, void* stream);

/* Case c's stored moments: rho[n], u[n][dim], T[n] (interior points: moments
 * of the last transported state; wall points: moments of f_b).  Host
 * destination (on_device = 0) is synchronous; device destination is
 * stream-ordered. */
int bgk_moments(bgk_ctx* ctx, int32_t c, double* rho, double* u, double* T, int32_t on_device, void* stream);

/* Case c's current positions x[n][dim] (host or device destination, as bgk_moments). */
int bgk_get_positions(bgk_ctx* ctx, int32_t c, double* x, int32_t on_device, void* stream);

/* Case c's current body centre, centre[dim] on the host (Sec. 3.4.1; the centre
 * advances with the body's points).  Synchronous (waits for the device).  Returns
 * BGK_E_INVAL when the case has no body (body_wall = 0). */
int bgk_get_body(bgk_ctx* ctx, int32_t c, double* centre);

/* Wait for the stream and return the first device-side error since the last
 * bgk_sync (then cleared), or BGK_OK. */
int bgk_sync(bgk_ctx* ctx, void* stream);

/* Checkpoint: the full state (positions, f, moments, body centre, step count)
 * of every case as one host blob.  bgk_get_state with blob == NULL stores the size
 * needed in *used.  Both calls are synchronous. */
int bgk_get_state(bgk_ctx* ctx, void* blob, size_t cap, size_t* used);
int bgk_set_state(bgk_ctx* ctx, const void* blob, size_t size);

/* Change the physical parameters of case c: kn, tau_mode, dt, wall_T, lid_u,
 * lid_wall, ale, guard and body_u (the wall tables are rebuilt); the geometry,
 * the body's wall id, centre and radius, the velocity grid, the storage and the
 * neighbour settings must stay the same (BGK_E_INVAL otherwise).  Synchronous. */
int bgk_set_params(bgk_ctx* ctx, int32_t c, const bgk_params* p);

/* Point management of case c between steps (Sec. 3.5.2, adding and removing
 * points), one pass on the current positions:
 *  - an interior point closer than rmin (absolute distance) to a wall point is
 *    removed (the wall point stays on the boundary);
 *  - remaining interior points that are each other's nearest remaining interior
 *    neighbour and closer than rmin are replaced by one point at their midpoint;
 *  - an interior point in neither case with fewer than min_nbrs neighbours gets a
 *    new interior point at x_i - (h/2) c/|c|, c the sum of its neighbour
 *    separations, when that position lies in [guard, 1 - guard]^dim (wrapped in a
 *    periodic box), outside the body's guard sphere and no point of N(i) + {i} is
 *    within rmin of it;
 *  - f at a new position is the linear WLS reconstruction there from N(i) + {i};
 *    the stored moments of every point are recomputed from f.
 * Surviving points keep their order (a merged pair keeps the smaller index);
 * added points follow in the order of the points that made them, up to the
 * capacity n + spare_points (later additions are dropped).  Point indices change:
 * host arrays of per-point data must be re-read.  counts (host, int64[3])
 * receives the new point count, the points removed (merged away or next to a
 * wall) and the points added.  Synchronous.  BGK_E_STATE for a proper velocity
 * slab. */
int bgk_manage(bgk_ctx* ctx, int32_t c, double rmin, int32_t min_nbrs, int64_t* counts, void* stream);

/* Objective of the current state of case c, not in the paper: the x-momentum flux
 * through the lid plane averaged over the lid points,
 * J = (1/|lid|) sum_{b in lid} sum_k v_x v_n g_b(v_k) dv^dim  (v_n the last velocity
 * component, normal to the lid; g = g1 in 2D, f in 3D).  J (device, one double) is
 * incremented by J; when lam is not NULL, lam += scale dJ/df.  lam has the internal
 * layout [n][ncomp][NVp] (NVp from bgk_get_stats) of the compute type: double
 * for BGK_F64 storage, float otherwise.  Stream-ordered.  BGK_E_STATE for a proper
 * velocity slab (as bgk_adjoint_step). */
int bgk_objective(bgk_ctx* ctx, int32_t c, double* J, void* lam, double scale, void* stream);

/* One step of the discrete adjoint of bgk_step for fixed points (ale = 0), not in
 * the paper: with the current state f^n of case c and lam_in = dJ/df^{n+1},
 * lam_out = (df^{n+1}/df^n)^T lam_in, and dtheta (device, 4 doubles) is
 * incremented by [dJ/du_lid (3 components), dJ/dKn] through this step.  The
 * vector-Jacobian product differentiates every sub-step of Sec. 3.2: the linear
 * upwind transport (transposed through the symmetric neighbour relation), the
 * relaxation through rho, U, T, tau(rho, T; Kn) and M, and the walls through the
 * reconstruction weights and the zero-mass-flux density rho_w, whose wall
 * Maxwellian depends on u_lid.  lam_in and lam_out are distinct device buffers
 * with the layout of bgk_objective.  The state f is not changed.  Work buffers
 * (three copies of f) are allocated on the first call.  Stream-ordered;
 * BGK_E_STATE when ale = 1. */
int bgk_adjoint_step(bgk_ctx* ctx, int32_t c, const void* lam_in, void* lam_out, double* dtheta, void* stream);

/* How bgk_step advances several cases (not in the paper, which steps one cavity):
 * mode 0 launches the kernels of each case in turn; mode 1 advances all cases
 * with one persistent transport launch over a (case, point) work list and one
 * wall launch over a (case, wall point) list; mode 2 replays those two launches
 * from a CUDA graph captured once per buffer parity.  Modes 1 and 2 apply when
 * every case is 2D with FP32 or BF16 storage (the same for all) and fixed points;
 * otherwise mode 0 is used.  mode = -1 (default) selects 2 for
 * n_cases > 1 and 0 otherwise.  The results are the same in every mode. */
int bgk_set_batching(bgk_ctx* ctx, int32_t mode);

/* Time the batched transport for CTA sizes of 4 and 8 warps and persistent grids
 * of {1, 2, 3, 4, 6} x the SM count (or one CTA per tile) on the current state and
 * keep the fastest (see bgk_stats).  The state is not changed.  Synchronous. */
int bgk_autotune(bgk_ctx* ctx, void* stream);

/* Per-kernel timing with CUDA events on the launching stream: bit k of enable
 * brackets every launch of kernel group k with an event pair (0 = transport+
 * relaxation, 1 = wall, 2 = neighbour build, 3 = stencils, 4 = motion, 5 = adjoint
 * step, 6 = one batched step of all cases; 0x7f times all, 0 none).  Each pair
 * costs the stream a little, so time only what is needed.  bgk_get_timing
 * synchronises and returns the summed device time (ms) and launch count of
 * group `which` since timing was enabled. */
int bgk_set_timing(bgk_ctx* ctx, int32_t enable);
int bgk_get_timing(bgk_ctx* ctx, int32_t which, double* total_ms, int64_t* launches);

int bgk_get_stats(bgk_ctx* ctx, bgk_stats* out);

/* One-line description of the last error on ctx (or of the last failed
 * bgk_init when ctx is NULL).  The string lives until the next call on ctx. */
const char* bgk_last_error(const bgk_ctx* ctx);

/* Release the context and all device memory it owns.  NULL is ignored. */
void bgk_free(bgk_ctx* ctx);

/* Neighbour lists for callers that cannot allocate device memory (code under a
 * memory manager that owns the device heap, or code that must not allocate
 * after start-up).  The paper has no counterpart: this is the neighbour search
 * of bgk_neighbours (same test, same ascending order, bit-identical lists)
 * written into caller-owned buffers, with no context and no allocation.
 *   x    device, [n][dim] double positions (unit box; minimum image if periodic)
 *   cnt  device, [n] int32 output: neighbours kept per point (<= cap)
 *   col  device, [n][cap] int32 output: neighbour indices, ascending per row
 * The cell-list scratch is a fixed array of about 3.7 MB in device global
 * memory, present on every GPU that loads the library until exit.  Limits:
 * n <= 131072 points, at most 131072 cells (cells per axis = floor(1/h)),
 * cap <= 443; larger sizes return BGK_E_INVAL without doing any work.  The
 * first call on a device looks up the array's address (make it before any
 * stream capture).  Every call clears what must start at zero; calls that
 * overlap on the GPU share the scratch and race.  Stream-ordered; with
 * check = 1 the call waits for the stream and returns BGK_E_NBR_OVERFLOW when
 * some point had more than cap neighbours (its row is then truncated). */
int bgk_neighbours_noalloc(int32_t dim, int64_t n, const double* x, double h, int32_t periodic,
                           int32_t cap, int32_t* cnt, int32_t* col, int32_t check, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BGK_H */
