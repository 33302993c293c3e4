// C ABI of libbgk (include/bgk.h): context, buffers, launch order of one time step.
//
// One time step of a case (Sec. 3.2, read in the order neighbours/stencils ->
// transport -> moments -> relaxation -> walls -> motion):
//   [ale or first step] cell lists, neighbour lists, WLS stencils
//   k_transport   f[cur] -> f[1-cur] at interior points (transport, moments, relaxation)
//   k_walls       f[1-cur] at wall points (reconstruction + diffuse reflection)
//   [ale]         k_move: x += dt U^{n+1}
// All launches go to the caller's stream; nothing synchronises inside bgk_step.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bgk.h"

// NVTX ranges (header-only NVTX 3; inert unless a profiler attaches): one per public
// call that launches work and one per launch group inside bgk_step, named by the group.
#ifndef BGK_NVTX
#define BGK_NVTX 1
#endif
#if BGK_NVTX
#include <nvtx3/nvToolsExt.h>
#define BGK_RANGE_PUSH(name) nvtxRangePushA(name)
#define BGK_RANGE_POP() nvtxRangePop()
#else
#define BGK_RANGE_PUSH(name) ((void)0)
#define BGK_RANGE_POP() ((void)0)
#endif

// Parts (and streams) of one staged upload (bgk_stage_f).
#ifndef BGK_UPLOAD_PARTS
#define BGK_UPLOAD_PARTS 4
#endif
#include "bgk_internal.cuh"

using namespace bgk;

namespace {

thread_local std::string g_init_error;

struct EvPair {
  cudaEvent_t a, b;
  int kid;
};

struct CaseHost {
  bgk_params p;
  CaseView cv;
  void* f[2];
  int cur;
  bool stencils_valid;
  size_t s_bytes, c_bytes;  // storage and compute element sizes
  // discrete adjoint (allocated on first use)
  void* adj_ft = nullptr;
  void* adj_y = nullptr;
  void* adj_lft = nullptr;
  double* adj_wmu = nullptr;
  double* adj_mom = nullptr;
  float* adj_sk = nullptr;
  int32_t* tslot = nullptr;
  int32_t* wall_of = nullptr;
  bool tslot_valid = false;
  int32_t nlid = 0;
  // velocity slab: a proper part of the grid (only the sharded calls step it); the
  // sharded step's next call (0 transport, 1 relax, 2 walls) and the side chain whose
  // wall weights its wall kernel waits for
  bool slab = false;
  int shard_phase = 0;
  int64_t shard_recon = -1;
  // caller-owned distribution storage (bgk_bind_f): it takes the place of f[bound_slot],
  // whose own buffer is kept in own_buf for the unbinding
  void* bound = nullptr;
  int bound_slot = -1;
  void* own_buf = nullptr;
  // input staged by bgk_stage_f for the next step: a third buffer filled on the copy
  // stream (ev_staged), swapped in by the next bgk_step, whose start (ev_free) frees the
  // buffer it replaces for the next upload
  void* staged = nullptr;
  bool staged_ready = false;
  bool free_recorded = false;
  cudaEvent_t ev_staged = nullptr, ev_free = nullptr;
  // ALE: the lists of the next step (second set of cnt, col, P, recon) are built on
  // the side stream right after the motion, while the wall kernel runs; they are
  // swapped in at the next step.  ev_fork orders the side work after the transport,
  // ev_join orders later work after it.
  int32_t* nx_cnt = nullptr;
  int32_t* nx_col = nullptr;
  void* nx_P = nullptr;
  void* nx_recon = nullptr;
  bool next_ready = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // wall reconstruction weights of the second set follow on the side stream while
  // the next transport runs; chain k records ev_recon[k & 1], which the wall kernel
  // of the step that uses that set waits for
  cudaEvent_t ev_recon[2] = {nullptr, nullptr};
  int64_t chain = 0;
  int chain_grid = 0;  // CTAs of the cooperative side-chain kernel (0: not yet sized)
  int64_t cap_n = 0;  // capacity of the per-point arrays (initial points + spare_points)
  // point management scratch (allocated on first use, cap_n entries)
  int32_t *pm_nn = nullptr, *pm_role = nullptr, *pm_newidx = nullptr, *pm_addidx = nullptr, *pm_totals = nullptr;
  int32_t *pm_kind2 = nullptr, *pm_int2 = nullptr;
  double *pm_ynew = nullptr, *pm_x2 = nullptr, *pm_norm2 = nullptr;
};

}  // namespace

struct bgk_ctx {
  std::vector<CaseHost> cases;
  // batched stepping of many cases (FP32/BF16, fixed points, one dimension)
  int batch_mode = -1;             // -1 default (graph when eligible and n_cases > 1), 0 per case, 1 batched, 2 batched + graph
  bool batch_ready = false;        // d_cases / items uploaded for the current parameters
  CaseView* d_cases[2] = {nullptr, nullptr};
  int2* d_items = nullptr;
  int2* d_witems = nullptr;
  int n_items = 0, n_witems = 0, capmax = 0, batch_dim = 0, batch_storage = 0;
  int batch_warps = 8, batch_grid = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side = nullptr;  // ALE motion and next-step lists, concurrent with the wall kernel
  cudaStream_t copy = nullptr;  // uploads of bgk_stage_f (the first part, and the join)
  // the other parts of an upload, each on a stream of its own so that several copy
  // engines take part; ev_part[k] joins part k + 1 back into copy
  cudaStream_t copy_part[BGK_UPLOAD_PARTS - 1] = {};
  cudaEvent_t ev_part[BGK_UPLOAD_PARTS - 1] = {};
  std::vector<void*> allocs;
  DevStatus* status = nullptr;
  std::string err;
  int64_t steps = 0, launches = 0;
  bool timing = false;
  int32_t timing_mask = 0;  // bit k: time kernel id k
  int64_t watchdog = 0;     // polls a bounded device wait makes before it gives up (0: default)
  std::vector<EvPair> ev;
  size_t ev_used = 0;
  double t_ms[K_COUNT] = {0, 0, 0, 0, 0, 0, 0};
  int64_t t_n[K_COUNT] = {0, 0, 0, 0, 0, 0, 0};
  void* staging = nullptr;
  size_t staging_bytes = 0;
};

namespace {

int fail(bgk_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_init_error = buf;
  return code;
}

#define CK(ctx, call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail((ctx), BGK_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKL(ctx)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess) return fail((ctx), BGK_E_CUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(bgk_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = count ? count * sizeof(T) : sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BGK_E_NOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  ctx->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return BGK_OK;
}

int dalloc_bytes(bgk_ctx* ctx, void** p, size_t bytes) {
  unsigned char* q = nullptr;
  int st = dalloc(ctx, &q, bytes);
  *p = q;
  return st;
}

int ensure_staging(bgk_ctx* ctx, size_t bytes) {
  if (ctx->staging_bytes >= bytes) return BGK_OK;
  if (ctx->staging) cudaFree(ctx->staging);
  ctx->staging = nullptr;
  ctx->staging_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->staging, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BGK_E_NOMEM, "staging cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->staging_bytes = bytes;
  return BGK_OK;
}

int check_params(const bgk_params& p, int64_t n, const char** why) {
  if (p.dim != 2 && p.dim != 3) { *why = "dim must be 2 or 3"; return 0; }
  if (p.nv < 2 || p.nv > 64) { *why = "nv must be in [2, 64]"; return 0; }
  int64_t NV = p.dim == 2 ? (int64_t)p.nv * p.nv : (int64_t)p.nv * p.nv * p.nv;
  if (NV > 8192) { *why = "nv^dim must be <= 8192"; return 0; }
  if (p.time_order < 0 || p.time_order > 2) { *why = "time_order must be 0, 1 or 2"; return 0; }
  if (p.vgrid < 0 || p.vgrid > 1) { *why = "vgrid must be 0 or 1"; return 0; }
  if (p.time_order == 2 && p.ale) { *why = "time_order 2 needs fixed points (ale = 0)"; return 0; }
  if (p.vk_hi == 0 ? p.vk_lo != 0 : (p.vk_lo < 0 || p.vk_lo >= p.vk_hi || p.vk_hi > NV || p.vk_lo % 4 != 0)) {
    *why = "velocity slab must satisfy 0 <= vk_lo < vk_hi <= nv^dim, vk_lo % 4 == 0 (or vk_lo = vk_hi = 0)";
    return 0;
  }
  if (!(p.vmax > 0) || !(p.dt > 0) || !(p.h > 0) || !(p.alpha > 0) || !(p.wall_T > 0)) {
    *why = "vmax, dt, h, alpha, wall_T must be positive";
    return 0;
  }
  if (p.tau_mode < 0 || p.tau_mode > 2) { *why = "tau_mode must be 0, 1 or 2"; return 0; }
  if (p.tau_mode != 2 && !(p.kn > 0)) { *why = "kn must be positive"; return 0; }
  if (p.storage < 0 || p.storage > 2) { *why = "storage must be 0 (f64), 1 (f32) or 2 (bf16)"; return 0; }
  if (p.max_nbrs < 1 || p.max_nbrs > 512) { *why = "max_nbrs must be in [1, 512]"; return 0; }
  if (n < 1 || n > (int64_t)1 << 30) { *why = "point count must be in [1, 2^30]"; return 0; }
  if (p.guard < 0 || p.guard >= 0.5) { *why = "guard must be in [0, 0.5)"; return 0; }
  if (!(p.skin >= 0 && p.skin <= 1)) { *why = "skin must be in [0, 1]"; return 0; }
  if (p.spare_points < 0 || n + p.spare_points > (int64_t)1 << 30) { *why = "spare_points out of range"; return 0; }
  if (p.wls_order < 0 || p.wls_order > 2) { *why = "wls_order must be 0, 1 or 2"; return 0; }
  if (p.body_wall < 0) { *why = "body_wall must be >= 0"; return 0; }
  if (p.body_wall > 0) {
    if (p.body_wall == p.lid_wall) { *why = "body_wall must differ from lid_wall"; return 0; }
    if (p.periodic) { *why = "a body needs a walled domain (periodic = 0)"; return 0; }
    if (!(p.body_radius >= 0) || !std::isfinite(p.body_radius)) { *why = "body_radius must be finite and >= 0"; return 0; }
    bool moving = false;
    for (int a = 0; a < 3; ++a) {
      if (!std::isfinite(p.body_u[a]) || !std::isfinite(p.body_centre[a])) {
        *why = "body_u and body_centre must be finite";
        return 0;
      }
      moving = moving || p.body_u[a] != 0.0;
    }
    if (moving && !p.ale) { *why = "a moving body (body_u != 0) needs ale = 1"; return 0; }
  }
  return 1;
}

void refresh_view(CaseHost& c) {
  c.cv.f_in = c.f[c.cur];
  c.cv.f_out = c.f[1 - c.cur];
}

// With caller-owned storage bound, a call that ends with the state in the context's own
// buffer copies it into the caller's (one device copy of the n current rows).
int settle_bound(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  if (!c.bound || c.cur == c.bound_slot) return BGK_OK;
  const size_t b = (size_t)c.cv.n * c.cv.ncomp * c.cv.NVp * c.s_bytes;
  CK(ctx, cudaMemcpyAsync(c.f[c.bound_slot], c.f[c.cur], b, cudaMemcpyDeviceToDevice, s));
  c.cur = c.bound_slot;
  refresh_view(c);
  return BGK_OK;
}

// NVTX range names of the launch groups (KernelId order)
const char* const kGroupName[K_COUNT] = {"transport", "walls", "neighbours", "stencils", "motion", "adjoint",
                                         "batched step"};

// RAII NVTX range for a public call
struct CallRange {
  explicit CallRange(const char* name) { BGK_RANGE_PUSH(name); }
  ~CallRange() { BGK_RANGE_POP(); }
};

int timed_begin(bgk_ctx* ctx, int kid, cudaStream_t s, EvPair** out) {
  *out = nullptr;
  BGK_RANGE_PUSH(kGroupName[kid]);
  if (!((ctx->timing_mask >> kid) & 1)) return BGK_OK;
  if (ctx->ev_used == ctx->ev.size()) {
    EvPair e;
    CK(ctx, cudaEventCreate(&e.a));
    CK(ctx, cudaEventCreate(&e.b));
    e.kid = kid;
    ctx->ev.push_back(e);
  }
  EvPair* e = &ctx->ev[ctx->ev_used++];
  e->kid = kid;
  CK(ctx, cudaEventRecord(e->a, s));
  *out = e;
  return BGK_OK;
}

int timed_end(bgk_ctx* ctx, EvPair* e, cudaStream_t s) {
  BGK_RANGE_POP();
  if (e) CK(ctx, cudaEventRecord(e->b, s));
  return BGK_OK;
}

int collect_timing(bgk_ctx* ctx) {
  for (size_t q = 0; q < ctx->ev_used; ++q) {
    EvPair& e = ctx->ev[q];
    CK(ctx, cudaEventSynchronize(e.b));
    float ms = 0.0f;
    CK(ctx, cudaEventElapsedTime(&ms, e.a, e.b));
    ctx->t_ms[e.kid] += ms;
    ctx->t_n[e.kid] += 1;
  }
  ctx->ev_used = 0;
  return BGK_OK;
}

// Forces a candidate rebuild at the next list build of an ALE case with skin lists.
int reset_skin(bgk_ctx* ctx, CaseHost& c) {
  if (!c.cv.sk) return BGK_OK;
  const SkinState s0 = {0u, 1, 0u, 0};
  CK(ctx, cudaMemcpy(c.cv.sk, &s0, sizeof(s0), cudaMemcpyHostToDevice));
  return BGK_OK;
}

// Neighbour lists and stencils of the current positions into the list arrays of v
// (part: as launch_stencils).
int build_lists_into(bgk_ctx* ctx, const CaseView& v, cudaStream_t s, int part = 0) {
  EvPair* e;
  int st;
  if ((st = timed_begin(ctx, K_NBR, s, &e))) return st;
  ctx->launches += v.ale && v.sk ? launch_neighbours_skin(v, s) : launch_neighbours(v, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  if ((st = timed_begin(ctx, K_STENCIL, s, &e))) return st;
  ctx->launches += launch_stencils(v, s, part);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  return BGK_OK;
}

// Orders stream s after the side-stream work of case c (motion, next lists, wall weights).
int join_side(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  if (c.ev_join) CK(ctx, cudaStreamWaitEvent(s, c.ev_join, 0));
  if (c.chain > 0) CK(ctx, cudaStreamWaitEvent(s, c.ev_recon[(c.chain - 1) & 1], 0));
  return BGK_OK;
}

int build_lists(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  int st;
  if ((st = join_side(ctx, c, s))) return st;
  if ((st = build_lists_into(ctx, c.cv, s))) return st;
  c.next_ready = false;
  c.stencils_valid = true;
  c.tslot_valid = false;
  return BGK_OK;
}

// After the transport of an ALE case on stream s: on the side stream, move the
// points and build the lists of the new positions into the second list set.  The
// next transport waits for the interior stencils (ev_join); the wall weights that
// follow overlap it (no kernel writes x or that set meanwhile) and the next wall
// kernel waits for them.
int move_and_prebuild(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  int st;
  EvPair* e;
  if (!ctx->side) CK(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  if (!c.ev_fork) {
    CK(ctx, cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&c.ev_recon[0], cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&c.ev_recon[1], cudaEventDisableTiming));
  }
  if (!c.nx_cnt) {
    const size_t n = c.cap_n, cap = c.cv.cap, dim = c.cv.dim;
    if ((st = dalloc(ctx, &c.nx_cnt, n))) return st;
    if ((st = dalloc(ctx, &c.nx_col, n * cap))) return st;
    if ((st = dalloc_bytes(ctx, &c.nx_P, n * cap * dim * dim * c.c_bytes))) return st;
    if ((st = dalloc_bytes(ctx, &c.nx_recon, n * cap * c.c_bytes))) return st;
    // empty rows until the first build fills them (a build cut short by a watchdog
    // timeout leaves the rows it did not reach as they were); on s, before ev_fork, so
    // that the side stream's build comes after it whatever stream s is
    CK(ctx, cudaMemsetAsync(c.nx_cnt, 0, sizeof(int32_t) * n, s));
  }
  cudaStream_t q = ctx->side;
  CK(ctx, cudaEventRecord(c.ev_fork, s));
  CK(ctx, cudaStreamWaitEvent(q, c.ev_fork, 0));
  CaseView nx = c.cv;
  nx.cnt = c.nx_cnt;
  nx.col = c.nx_col;
  nx.P = c.nx_P;
  nx.recon = c.nx_recon;
  if (chain_eligible(nx)) {
    // motion, lists and interior stencils in one cooperative launch (timed as lists)
    if ((st = timed_begin(ctx, K_NBR, q, &e))) return st;
    const int k = launch_chain(nx, &c.chain_grid, ctx->watchdog, q);
    if (k < 0) return fail(ctx, BGK_E_CUDA, "cooperative launch of the side chain failed");
    ctx->launches += k;
    CKL(ctx);
    if ((st = timed_end(ctx, e, q))) return st;
  } else {
    if ((st = timed_begin(ctx, K_MOVE, q, &e))) return st;
    ctx->launches += launch_move(c.cv, q);
    CKL(ctx);
    if ((st = timed_end(ctx, e, q))) return st;
    if ((st = build_lists_into(ctx, nx, q, 1))) return st;
  }
  CK(ctx, cudaEventRecord(c.ev_join, q));
  if ((st = timed_begin(ctx, K_STENCIL, q, &e))) return st;
  ctx->launches += launch_stencils(nx, q, 2);
  CKL(ctx);
  if ((st = timed_end(ctx, e, q))) return st;
  CK(ctx, cudaEventRecord(c.ev_recon[c.chain & 1], q));
  c.chain += 1;
  c.next_ready = true;
  return BGK_OK;
}

// At the start of a step: the lists built after the last motion become current.
void swap_in_next(CaseHost& c) {
  std::swap(c.cv.cnt, c.nx_cnt);
  std::swap(c.cv.col, c.nx_col);
  std::swap(c.cv.P, c.nx_P);
  std::swap(c.cv.recon, c.nx_recon);
  c.next_ready = false;
  c.tslot_valid = false;
}

// ---- batched stepping ----

bool batch_eligible(const bgk_ctx* ctx) {
  if (ctx->cases.empty()) return false;
  const CaseHost& c0 = ctx->cases[0];
  if (c0.cv.dim != 2) return false;  // the batched kernels are the 2D ones
  for (const CaseHost& c : ctx->cases) {
    if (c.slab || c.p.time_order == 2 || c.cv.ale || c.p.storage == 0 || c.p.storage != c0.p.storage || c.cv.dim != c0.cv.dim || c.cur != c0.cur)
      return false;
  }
  return true;
}

int effective_mode(const bgk_ctx* ctx) {
  if (!batch_eligible(ctx)) return 0;
  if (ctx->batch_mode >= 0) return ctx->batch_mode;
  return ctx->cases.size() > 1 ? 2 : 0;
}

void drop_graphs(bgk_ctx* ctx) {
  for (int q = 0; q < 2; ++q)
    if (ctx->graph[q]) {
      cudaGraphExecDestroy(ctx->graph[q]);
      ctx->graph[q] = nullptr;
    }
}

void invalidate_batch(bgk_ctx* ctx) {
  ctx->batch_ready = false;
  drop_graphs(ctx);
}

// Upload the per-parity case descriptors and the (case, slot) work lists.
int prepare_batch(bgk_ctx* ctx, cudaStream_t s) {
  if (ctx->batch_ready) return BGK_OK;
  int st;
  for (auto& c : ctx->cases) {
    refresh_view(c);
    if (!c.stencils_valid && (st = build_lists(ctx, c, s))) return st;
  }
  const int nc = (int)ctx->cases.size();
  if (!ctx->d_cases[0]) {
    for (int q = 0; q < 2; ++q)
      if ((st = dalloc(ctx, &ctx->d_cases[q], nc))) return st;
    std::vector<int2> items, witems;
    int capmax = 0;
    for (int ci = 0; ci < nc; ++ci) {
      const CaseView& v = ctx->cases[ci].cv;
      for (int k = 0; k < v.n_int; ++k) items.push_back(make_int2(ci, k));
      for (int k = 0; k < v.n_wall; ++k) witems.push_back(make_int2(ci, k));
      capmax = std::max(capmax, v.cap);
    }
    if ((st = dalloc(ctx, &ctx->d_items, std::max<size_t>(items.size(), 1)))) return st;
    if ((st = dalloc(ctx, &ctx->d_witems, std::max<size_t>(witems.size(), 1)))) return st;
    CK(ctx, cudaMemcpy(ctx->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->d_witems, witems.data(), sizeof(int2) * witems.size(), cudaMemcpyHostToDevice));
    ctx->n_items = (int)items.size();
    ctx->n_witems = (int)witems.size();
    ctx->capmax = capmax;
    ctx->batch_dim = ctx->cases[0].cv.dim;
    ctx->batch_storage = ctx->cases[0].p.storage;
  }
  std::vector<CaseView> views(nc);
  for (int q = 0; q < 2; ++q) {
    for (int ci = 0; ci < nc; ++ci) {
      CaseHost& c = ctx->cases[ci];
      views[ci] = c.cv;
      views[ci].f_in = c.f[q];
      views[ci].f_out = c.f[1 - q];
    }
    CK(ctx, cudaMemcpyAsync(ctx->d_cases[q], views.data(), sizeof(CaseView) * nc, cudaMemcpyHostToDevice, s));
  }
  CK(ctx, cudaStreamSynchronize(s));
  ctx->batch_ready = true;
  return BGK_OK;
}

int launch_batch_step(bgk_ctx* ctx, int parity, cudaStream_t s) {
  ctx->launches += launch_transport_batch(ctx->d_cases[parity], ctx->d_items, ctx->n_items, ctx->batch_dim,
                                          ctx->batch_storage, ctx->capmax, ctx->batch_warps, ctx->batch_grid, s);
  ctx->launches += launch_walls_batch(ctx->d_cases[parity], ctx->d_witems, ctx->n_witems, ctx->batch_dim,
                                      ctx->batch_storage, ctx->capmax, s);
  CKL(ctx);
  return BGK_OK;
}

int capture_graphs(bgk_ctx* ctx) {
  if (ctx->graph[0] && ctx->graph[1]) return BGK_OK;
  if (!ctx->cap_stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  for (int q = 0; q < 2; ++q) {
    cudaGraph_t g = nullptr;
    CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = ctx->launches;
    int st = launch_batch_step(ctx, q, ctx->cap_stream);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->launches = l0;  // counted when the graph is launched
    if (st) return st;
    if (e != cudaSuccess) return fail(ctx, BGK_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph[q], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, BGK_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return BGK_OK;
}

}  // namespace

extern "C" {

int bgk_version(void) { return BGK_ABI_VERSION; }

int bgk_init(const bgk_params* p, int32_t n_cases, const int64_t* n_points, const double* x,
             const int32_t* kind, const double* normal, bgk_ctx** out) {
  if (!out) return fail(nullptr, BGK_E_INVAL, "bgk_init: out is NULL");
  *out = nullptr;
  if (!p || !n_points || !x || !kind || !normal || n_cases < 1)
    return fail(nullptr, BGK_E_INVAL, "bgk_init: NULL argument or n_cases < 1");
  for (int c = 0; c < n_cases; ++c) {
    const char* why = nullptr;
    if (!check_params(p[c], n_points[c], &why)) return fail(nullptr, BGK_E_INVAL, "bgk_init: case %d: %s", c, why);
  }
  // geometry: positions finite and inside the unit box that the cell grid spans, kinds
  // >= 0, normals finite (the arrays are read with the offsets of the copies below)
  {
    int64_t off = 0;
    for (int c = 0; c < n_cases; ++c) {
      const int dim = p[c].dim;
      for (int64_t k = off; k < off + n_points[c]; ++k) {
        for (int a = 0; a < dim; ++a) {
          const double xa = x[k * dim + a], na = normal[k * dim + a];
          if (!(xa >= 0.0 && xa <= 1.0))
            return fail(nullptr, BGK_E_INVAL, "bgk_init: case %d: point %lld: coordinate %d = %g is not in [0, 1]",
                        c, (long long)(k - off), a, xa);
          if (!std::isfinite(na))
            return fail(nullptr, BGK_E_INVAL, "bgk_init: case %d: point %lld: normal is not finite", c,
                        (long long)(k - off));
        }
        if (kind[k] < 0) return fail(nullptr, BGK_E_INVAL, "bgk_init: case %d: point %lld: kind < 0", c, (long long)(k - off));
      }
      off += n_points[c];
    }
  }
  bgk_ctx* ctx = new (std::nothrow) bgk_ctx();
  if (!ctx) return fail(nullptr, BGK_E_NOMEM, "bgk_init: host allocation failed");
  int st = BGK_OK;
  auto bail = [&](int code) {
    g_init_error = ctx->err;
    bgk_free(ctx);
    return code;
  };
  if ((st = dalloc(ctx, &ctx->status, 1))) return bail(st);
  if (cudaMemset(ctx->status, 0, sizeof(DevStatus)) != cudaSuccess) return bail(fail(ctx, BGK_E_CUDA, "cudaMemset status"));
  int64_t off = 0;
  ctx->cases.resize(n_cases);
  for (int ci = 0; ci < n_cases; ++ci) {
    CaseHost& c = ctx->cases[ci];
    const bgk_params& q = p[ci];
    const int64_t n = n_points[ci];
    const int dim = q.dim;
    c.p = q;
    c.cur = 0;
    c.stencils_valid = false;
    CaseView& v = c.cv;
    memset(&v, 0, sizeof(v));
    v.dim = dim;
    v.nv = q.nv;
    v.NV = dim == 2 ? q.nv * q.nv : q.nv * q.nv * q.nv;
    if (q.vk_hi > 0) {
      c.slab = q.vk_lo != 0 || q.vk_hi != v.NV;
      v.vk0 = q.vk_lo;
      v.NV = q.vk_hi - q.vk_lo;
    }
    v.NVp = (v.NV + 3) / 4 * 4;
    v.ncomp = dim == 2 ? 2 : 1;
    v.cap = q.max_nbrs;
    v.n = (int32_t)n;
    v.ale = q.ale;
    v.periodic = q.periodic;
    v.tau_mode = q.tau_mode;
    v.lid_wall = q.lid_wall;
    v.storage = q.storage;
    v.dt = q.dt;
    v.h = q.h;
    v.alpha = q.alpha;
    v.kn = q.kn;
    v.wall_T = q.wall_T;
    v.guard = q.guard;
    v.dv = q.vgrid == 1 ? 2.0 * q.vmax / (double)q.nv : 2.0 * q.vmax / (double)(q.nv - 1);
    set_case_consts(v);
    for (int a = 0; a < 3; ++a) v.lid_u[a] = q.lid_u[a];
    v.skin = q.skin;
    v.body_wall = q.body_wall;
    for (int a = 0; a < 3; ++a) v.body_u[a] = q.body_u[a];
    v.body_rg = q.body_radius + q.guard;
    v.wls_order = q.wls_order;
    // cells of side >= the search radius (h, or h (1 + skin) for the candidate lists)
    v.nc = (int)std::floor(1.0 / (q.h * (1.0 + q.skin) * (1.0 + 1e-9)));
    if (v.nc < 1) v.nc = 1;
    if (v.nc > 4096) v.nc = 4096;
    int64_t ncell = 1;
    for (int a = 0; a < dim; ++a) ncell *= v.nc;
    if (ncell > (int64_t)1 << 26) return bail(fail(ctx, BGK_E_INVAL, "case %d: too many cells (h too small)", ci));
    v.ncell = (int32_t)ncell;
    c.s_bytes = q.storage == 0 ? 8 : (q.storage == 1 ? 4 : 2);
    c.c_bytes = q.storage == 0 ? 8 : 4;

    // interior / wall partition of the input.  Interior points are listed in Morton
    // (Z) order of their initial positions, so that consecutive points (the points of
    // one CTA) are spatially compact and share most of their neighbours; wall points
    // are listed in index order.  The order changes which CTA handles a point, not
    // its arithmetic.
    std::vector<int32_t> inner, wall;
    std::vector<std::pair<uint64_t, int32_t>> keyed;
    for (int64_t i = 0; i < n; ++i) {
      if (kind[off + i] != 0) { wall.push_back((int32_t)i); continue; }
      uint64_t key = 0;
      for (int a = 0; a < dim; ++a) {
        double xa = x[(off + i) * dim + a];
        xa = xa < 0.0 ? 0.0 : (xa > 1.0 ? 1.0 : xa);
        const uint64_t qa = (uint64_t)(xa * 1048575.0);  // 20 bits per axis
        for (int bit = 0; bit < 20; ++bit) key |= ((qa >> bit) & 1ull) << (bit * dim + a);
      }
      keyed.emplace_back(key, (int32_t)i);
    }
    std::sort(keyed.begin(), keyed.end());
    for (auto& kv : keyed) inner.push_back(kv.second);
    if (q.periodic && !wall.empty()) return bail(fail(ctx, BGK_E_INVAL, "case %d: periodic box with wall points", ci));
    v.n_int = (int32_t)inner.size();
    v.n_wall = (int32_t)wall.size();
    c.nlid = 0;
    for (int64_t i = 0; i < n; ++i) c.nlid += kind[off + i] == q.lid_wall && q.lid_wall != 0;
    // per-point arrays hold cap_n = n + spare_points points (room for added points)
    const int64_t ncap = n + q.spare_points;
    c.cap_n = ncap;
    std::vector<int32_t> wall_of(n, -1);
    for (size_t w = 0; w < wall.size(); ++w) wall_of[wall[w]] = (int32_t)w;
    if ((st = dalloc(ctx, &c.wall_of, ncap))) return bail(st);
    if (cudaMemcpy(c.wall_of, wall_of.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, BGK_E_CUDA, "case %d: wall map upload failed", ci));

    double* dx = nullptr;
    int32_t *dkind = nullptr, *dint = nullptr, *dwall = nullptr;
    double* dnorm = nullptr;
    if ((st = dalloc(ctx, &dx, ncap * dim))) return bail(st);
    if ((st = dalloc(ctx, &dkind, ncap))) return bail(st);
    if ((st = dalloc(ctx, &dnorm, ncap * dim))) return bail(st);
    if ((st = dalloc(ctx, &dint, inner.size() + q.spare_points))) return bail(st);
    if ((st = dalloc(ctx, &dwall, wall.size()))) return bail(st);
    if (cudaMemcpy(dx, x + off * dim, sizeof(double) * n * dim, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dkind, kind + off, sizeof(int32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dnorm, normal + off * dim, sizeof(double) * n * dim, cudaMemcpyHostToDevice) != cudaSuccess ||
        (inner.size() && cudaMemcpy(dint, inner.data(), sizeof(int32_t) * inner.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        (wall.size() && cudaMemcpy(dwall, wall.data(), sizeof(int32_t) * wall.size(), cudaMemcpyHostToDevice) != cudaSuccess))
      return bail(fail(ctx, BGK_E_CUDA, "case %d: geometry upload failed", ci));
    v.x = dx;
    v.kind = dkind;
    v.normal = dnorm;
    v.int_idx = dint;
    v.wall_idx = dwall;

    if ((st = dalloc(ctx, &v.vnodes, q.nv))) return bail(st);
    if ((st = dalloc(ctx, &v.vnodes_f, q.nv))) return bail(st);
    if ((st = dalloc(ctx, &v.xf, ncap * dim))) return bail(st);
    if ((st = dalloc(ctx, &v.xlo, ncap * dim))) return bail(st);
    if ((st = dalloc(ctx, &v.cell_of, ncap))) return bail(st);
    if ((st = dalloc(ctx, &v.cell_start, ncell + 1))) return bail(st);
    if ((st = dalloc(ctx, &v.cell_cnt, ncell))) return bail(st);
    if ((st = dalloc(ctx, &v.cell_pts, ncap))) return bail(st);
    if ((st = dalloc(ctx, &v.cnt, ncap))) return bail(st);
    if ((st = dalloc(ctx, &v.col, ncap * v.cap))) return bail(st);
    if ((st = dalloc_bytes(ctx, &v.P, (size_t)ncap * v.cap * dim * dim * c.c_bytes))) return bail(st);
    if ((st = dalloc_bytes(ctx, &v.recon, (size_t)ncap * v.cap * c.c_bytes))) return bail(st);
    if ((st = dalloc(ctx, &v.wcls, (size_t)v.n_wall * v.NVp))) return bail(st);
    if ((st = dalloc_bytes(ctx, &v.wvn, (size_t)v.n_wall * v.NVp * c.c_bytes))) return bail(st);
    if ((st = dalloc(ctx, &v.winv, v.n_wall))) return bail(st);
    if ((st = dalloc_bytes(ctx, &v.mw, (size_t)3 * v.NVp * c.c_bytes))) return bail(st);
    if (q.body_wall > 0) {
      if ((st = dalloc(ctx, &v.body, 1))) return bail(st);
      BodyState b0;
      memset(&b0, 0, sizeof(b0));
      for (int a = 0; a < dim; ++a) b0.c[a] = q.body_centre[a];
      if (cudaMemcpy(v.body, &b0, sizeof(b0), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(ctx, BGK_E_CUDA, "case %d: body state upload failed", ci));
    }
    const size_t fbytes = (size_t)ncap * v.ncomp * v.NVp * c.s_bytes;
    for (int b = 0; b < 2; ++b) {
      if ((st = dalloc_bytes(ctx, &c.f[b], fbytes))) return bail(st);
      if (cudaMemset(c.f[b], 0, fbytes) != cudaSuccess) return bail(fail(ctx, BGK_E_CUDA, "cudaMemset f"));
    }
    if (q.skin > 0) {
      // candidate capacity: max_nbrs scaled by the volume ratio of the two radii, plus 10 %
      const double r = std::pow(1.0 + q.skin, dim) * 1.1;
      v.ccap = (int32_t)std::min<double>(std::ceil(v.cap * r), 4096.0);
      if ((st = dalloc(ctx, &v.xb, ncap * dim))) return bail(st);
      if ((st = dalloc(ctx, &v.ccnt, ncap))) return bail(st);
      if ((st = dalloc(ctx, &v.ccol, (size_t)ncap * v.ccap))) return bail(st);
      if ((st = dalloc(ctx, &v.sk, 1))) return bail(st);
      const SkinState s0 = {0u, 1, 0u, 0};
      if (cudaMemcpy(v.sk, &s0, sizeof(s0), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemset(v.cell_cnt, 0, sizeof(int32_t) * ncell) != cudaSuccess)
        return bail(fail(ctx, BGK_E_CUDA, "case %d: skin state upload failed", ci));
    }
    if ((st = dalloc(ctx, &v.mom, (size_t)ncap * MOM_STRIDE))) return bail(st);
    if (cudaMemset(v.mom, 0, sizeof(double) * ncap * MOM_STRIDE) != cudaSuccess) return bail(fail(ctx, BGK_E_CUDA, "cudaMemset mom"));
    v.status = ctx->status;
    refresh_view(c);
    ctx->launches += launch_init_tables(v, 0);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return bail(fail(ctx, BGK_E_CUDA, "case %d: table initialisation failed", ci));
    off += n;
  }
  DevStatus hs;
  if (cudaMemcpy(&hs, ctx->status, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bail(fail(ctx, BGK_E_CUDA, "status read failed"));
  if (hs.flags & ST_SINGULAR) return bail(fail(ctx, BGK_E_SINGULAR, "a wall point has no leaving velocity with positive flux"));
  *out = ctx;
  return BGK_OK;
}

int bgk_set_maxwellian(bgk_ctx* ctx, double rho0, const double* u0, double T0, void* stream) {
  if (!ctx || !u0) return BGK_E_INVAL;
  if (!(rho0 > 0) || !(T0 > 0)) return fail(ctx, BGK_E_INVAL, "bgk_set_maxwellian: rho0 and T0 must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  for (auto& c : ctx->cases) {
    refresh_view(c);
    ctx->launches += launch_set_maxwellian(c.cv, rho0, u0, T0, s);
    if (!c.slab) ctx->launches += launch_moments(c.cv, c.f[c.cur], s);
    CKL(ctx);
  }
  return BGK_OK;
}

int bgk_set_f(bgk_ctx* ctx, int32_t ci, const void* f, int32_t dtype, int32_t on_device, void* stream) {
  CallRange range_("bgk_set_f");
  if (!ctx || !f || ci < 0 || ci >= (int)ctx->cases.size() || dtype < 0 || dtype > 2)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_set_f: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  refresh_view(c);
  const size_t esz = dtype == 0 ? 8 : (dtype == 1 ? 4 : 2);
  const size_t bytes = (size_t)c.cv.n * c.cv.ncomp * c.cv.NV * esz;
  const void* src = f;
  const bool direct = dtype == c.cv.storage && c.cv.NV == c.cv.NVp;  // same element type, no padding
  if (on_device && direct && f == c.f[c.cur]) {
    // the bound storage itself, written by the caller: only the moments are recomputed
  } else if (!on_device && direct) {
    CK(ctx, cudaMemcpyAsync(c.f[c.cur], f, bytes, cudaMemcpyHostToDevice, s));
  } else {
    if (!on_device) {
      int st = ensure_staging(ctx, bytes);
      if (st) return st;
      CK(ctx, cudaMemcpyAsync(ctx->staging, f, bytes, cudaMemcpyHostToDevice, s));
      src = ctx->staging;
    }
    ctx->launches += launch_pack_f(c.cv, src, dtype, c.f[c.cur], s);
  }
  if (!c.slab) ctx->launches += launch_moments(c.cv, c.f[c.cur], s);
  CKL(ctx);
  if (!on_device) CK(ctx, cudaStreamSynchronize(s));
  return BGK_OK;
}

int bgk_get_f(bgk_ctx* ctx, int32_t ci, void* f, int32_t dtype, int32_t on_device, void* stream) {
  if (!ctx || !f || ci < 0 || ci >= (int)ctx->cases.size() || dtype < 0 || dtype > 2)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_get_f: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  refresh_view(c);
  const size_t esz = dtype == 0 ? 8 : (dtype == 1 ? 4 : 2);
  const size_t bytes = (size_t)c.cv.n * c.cv.ncomp * c.cv.NV * esz;
  if (on_device) {
    ctx->launches += launch_unpack_f(c.cv, c.f[c.cur], f, dtype, s);
    CKL(ctx);
    return BGK_OK;
  }
  if (dtype == c.cv.storage && c.cv.NV == c.cv.NVp) {  // same element type, no padding: direct copy
    CK(ctx, cudaMemcpyAsync(f, c.f[c.cur], bytes, cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    return BGK_OK;
  }
  int st = ensure_staging(ctx, bytes);
  if (st) return st;
  ctx->launches += launch_unpack_f(c.cv, c.f[c.cur], ctx->staging, dtype, s);
  CKL(ctx);
  CK(ctx, cudaMemcpyAsync(f, ctx->staging, bytes, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  return BGK_OK;
}

int bgk_neighbours(bgk_ctx* ctx, void* stream) {
  CallRange range_("bgk_neighbours");
  if (!ctx) return BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  invalidate_batch(ctx);
  for (auto& c : ctx->cases) {
    refresh_view(c);
    int st = build_lists(ctx, c, s);
    if (st) return st;
  }
  return BGK_OK;
}

int bgk_get_neighbours(bgk_ctx* ctx, int32_t ci, int64_t* rowptr, int32_t* col, int64_t cap, int64_t* nnz) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || !rowptr || !nnz)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_get_neighbours: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  CK(ctx, cudaDeviceSynchronize());
  const int n = c.cv.n, K = c.cv.cap;
  std::vector<int32_t> cnt(n), ell((size_t)n * K);
  CK(ctx, cudaMemcpy(cnt.data(), c.cv.cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  CK(ctx, cudaMemcpy(ell.data(), c.cv.col, sizeof(int32_t) * ell.size(), cudaMemcpyDeviceToHost));
  int64_t z = 0;
  rowptr[0] = 0;
  for (int i = 0; i < n; ++i) { z += cnt[i]; rowptr[i + 1] = z; }
  *nnz = z;
  if (!col) return BGK_OK;
  if (cap < z) return fail(ctx, BGK_E_INVAL, "bgk_get_neighbours: cap %lld < nnz %lld", (long long)cap, (long long)z);
  for (int i = 0; i < n; ++i) memcpy(col + rowptr[i], ell.data() + (size_t)i * K, sizeof(int32_t) * cnt[i]);
  return BGK_OK;
}

int bgk_get_stencils(bgk_ctx* ctx, int32_t ci, double* P, double* recon, int64_t cap) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || !P || !recon)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_get_stencils: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  CK(ctx, cudaDeviceSynchronize());
  const int n = c.cv.n, dd = c.cv.dim * c.cv.dim;
  std::vector<int32_t> cnt(n);
  CK(ctx, cudaMemcpy(cnt.data(), c.cv.cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  std::vector<int64_t> rp(n + 1, 0);
  for (int i = 0; i < n; ++i) rp[i + 1] = rp[i] + cnt[i];
  const int64_t z = rp[n];
  if (cap < z) return fail(ctx, BGK_E_INVAL, "bgk_get_stencils: cap %lld < nnz %lld", (long long)cap, (long long)z);
  int64_t* drp = nullptr;
  double *dP = nullptr, *dR = nullptr;
  CK(ctx, cudaMalloc(&drp, sizeof(int64_t) * (n + 1)));
  CK(ctx, cudaMalloc(&dP, sizeof(double) * std::max<int64_t>(z, 1) * dd));
  CK(ctx, cudaMalloc(&dR, sizeof(double) * std::max<int64_t>(z, 1)));
  cudaMemcpy(drp, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
  ctx->launches += launch_stencils_csr(c.cv, drp, dP, dR, 0);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(P, dP, sizeof(double) * z * dd, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(recon, dR, sizeof(double) * z, cudaMemcpyDeviceToHost);
  cudaFree(drp);
  cudaFree(dP);
  cudaFree(dR);
  if (e != cudaSuccess) return fail(ctx, BGK_E_CUDA, "bgk_get_stencils: %s", cudaGetErrorString(e));
  return BGK_OK;
}

// One second-order step of a fixed-point case, f^{n+1} = R(dt/2) T(dt) R(dt/2) f^n, with
// A = f[cur] and B = f[1 - cur]: R(dt/2) on A in place; T1: A -> B (no relaxation) and
// the walls of B; T1 from B averaged with A and R(dt/2), into A; the walls of A.  The
// result stays in A.
static int step_second_order(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  int st;
  EvPair* e;
  CaseView a = c.cv;  // f_in = A, f_out = B
  CaseView pre = a;
  pre.f_out = a.f_in;
  CaseView s1 = a;
  s1.tau_mode = 2;
  CaseView s2 = a;
  s2.f_in = a.f_out;
  s2.f_out = a.f_in;
  s2.f_avg = a.f_in;
  if ((st = timed_begin(ctx, K_TRANSPORT, s, &e))) return st;
  ctx->launches += launch_relax_half(pre, s);
  ctx->launches += launch_transport(s1, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  if ((st = timed_begin(ctx, K_WALLS, s, &e))) return st;
  ctx->launches += launch_walls(s1, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  if ((st = timed_begin(ctx, K_TRANSPORT, s, &e))) return st;
  ctx->launches += launch_transport_avg(s2, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  if ((st = timed_begin(ctx, K_WALLS, s, &e))) return st;
  ctx->launches += launch_walls(s2, s);
  CKL(ctx);
  return timed_end(ctx, e, s);
}

// The input staged by bgk_stage_f becomes the state: stream s waits for its upload, the
// buffers are swapped, the moments are taken, and ev_free marks the point after which the
// replaced buffer (the next staging target) is no longer used.
static int take_staged(bgk_ctx* ctx, CaseHost& c, cudaStream_t s) {
  if (!c.staged_ready) return BGK_OK;
  CK(ctx, cudaStreamWaitEvent(s, c.ev_staged, 0));
  std::swap(c.f[c.cur], c.staged);
  refresh_view(c);
  ctx->launches += launch_moments(c.cv, c.f[c.cur], s);
  CKL(ctx);
  CK(ctx, cudaEventRecord(c.ev_free, s));
  c.free_recorded = true;
  c.staged_ready = false;
  invalidate_batch(ctx);
  return BGK_OK;
}

int bgk_step(bgk_ctx* ctx, int32_t nsteps, void* stream) {
  CallRange range_("bgk_step");
  if (!ctx || nsteps < 0) return ctx ? fail(ctx, BGK_E_INVAL, "bgk_step: nsteps < 0") : BGK_E_INVAL;
  for (const CaseHost& c : ctx->cases)
    if (c.slab) return fail(ctx, BGK_E_STATE, "bgk_step: a case holds a velocity slab (step it with bgk_shard_*)");
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  for (auto& c : ctx->cases)
    if ((st = take_staged(ctx, c, s))) return st;
  EvPair* e;
  const int mode = effective_mode(ctx);
  if (mode >= 1 && nsteps > 0) {
    if ((st = prepare_batch(ctx, s))) return st;
    if (mode == 2 && (st = capture_graphs(ctx))) return st;
    for (int step = 0; step < nsteps; ++step) {
      const int parity = ctx->cases[0].cur;
      if ((st = timed_begin(ctx, K_BATCH, s, &e))) return st;
      if (mode == 2) {
        CK(ctx, cudaGraphLaunch(ctx->graph[parity], s));
        ctx->launches += 2;
      } else if ((st = launch_batch_step(ctx, parity, s))) {
        return st;
      }
      if ((st = timed_end(ctx, e, s))) return st;
      for (auto& c : ctx->cases) {
        c.cur = 1 - c.cur;
        refresh_view(c);
      }
      ctx->steps += 1;
    }
    for (auto& c : ctx->cases)
      if ((st = settle_bound(ctx, c, s))) return st;
    return BGK_OK;
  }
  for (int step = 0; step < nsteps; ++step) {
    for (auto& c : ctx->cases) {
      refresh_view(c);
      int64_t recon_chain = -1;  // side chain whose wall weights the wall kernel needs
      if (c.next_ready && c.stencils_valid && c.cv.ale) {
        swap_in_next(c);
        CK(ctx, cudaStreamWaitEvent(s, c.ev_join, 0));
        recon_chain = c.chain - 1;
      } else if (c.cv.ale || !c.stencils_valid) {
        if ((st = build_lists(ctx, c, s))) return st;
      }
      if (c.p.time_order == 2) {
        if ((st = step_second_order(ctx, c, s))) return st;
        continue;
      }
      if ((st = timed_begin(ctx, K_TRANSPORT, s, &e))) return st;
      ctx->launches += launch_transport(c.cv, s);
      CKL(ctx);
      if ((st = timed_end(ctx, e, s))) return st;
      // ALE: motion and the next step's lists on the side stream (they read U^{n+1}
      // and write x and the second list set, which the wall kernel does not touch)
      if (c.cv.ale && (st = move_and_prebuild(ctx, c, s))) return st;
      if (recon_chain >= 0) CK(ctx, cudaStreamWaitEvent(s, c.ev_recon[recon_chain & 1], 0));
      if ((st = timed_begin(ctx, K_WALLS, s, &e))) return st;
      ctx->launches += launch_walls(c.cv, s);
      CKL(ctx);
      if ((st = timed_end(ctx, e, s))) return st;
      c.cur = 1 - c.cur;
      refresh_view(c);
    }
    ctx->steps += 1;
  }
  for (auto& c : ctx->cases) {
    if (c.next_ready && (st = join_side(ctx, c, s))) return st;
    if ((st = settle_bound(ctx, c, s))) return st;
  }
  return BGK_OK;
}

// ---- velocity-sharded step ----

// Case ci of a sharded call; buf (an exchange buffer) may be null only where the case
// has no wall points and the buffer is the wall sums.
static int shard_case(bgk_ctx* ctx, int32_t ci, const void* buf, bool wall_buf, const char* fn, CaseHost** out) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || (!buf && !(wall_buf && ctx->cases[ci].cv.n_wall == 0)))
    return ctx ? fail(ctx, BGK_E_INVAL, "%s: bad argument", fn) : BGK_E_INVAL;
  *out = &ctx->cases[ci];
  refresh_view(**out);
  return BGK_OK;
}

int bgk_shard_sizes(bgk_ctx* ctx, int32_t ci, int64_t* n_xm, int64_t* n_xw) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || !n_xm || !n_xw)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_shard_sizes: bad argument") : BGK_E_INVAL;
  const CaseView& v = ctx->cases[ci].cv;
  *n_xm = (int64_t)v.n * (v.dim + 2);
  *n_xw = (int64_t)v.n_wall * (2 * v.dim + 6);
  return BGK_OK;
}

int bgk_shard_transport(bgk_ctx* ctx, int32_t ci, double* xm, void* stream) {
  CallRange range_("bgk_shard_transport");
  CaseHost* cp = nullptr;
  int st;
  if ((st = shard_case(ctx, ci, xm, false, "bgk_shard_transport", &cp))) return st;
  CaseHost& c = *cp;
  if (c.shard_phase != 0) return fail(ctx, BGK_E_STATE, "bgk_shard_transport: the previous sharded step is not finished");
  if (c.p.time_order == 2) return fail(ctx, BGK_E_STATE, "bgk_shard_transport: not available with time_order 2");
  cudaStream_t s = (cudaStream_t)stream;
  invalidate_batch(ctx);
  // the lists of this step, as in bgk_step
  c.shard_recon = -1;
  if (c.next_ready && c.stencils_valid && c.cv.ale) {
    swap_in_next(c);
    CK(ctx, cudaStreamWaitEvent(s, c.ev_join, 0));
    c.shard_recon = c.chain - 1;
  } else if (c.cv.ale || !c.stencils_valid) {
    if ((st = build_lists(ctx, c, s))) return st;
  }
  EvPair* e;
  CaseView v = c.cv;
  v.xs = xm;
  if ((st = timed_begin(ctx, K_TRANSPORT, s, &e))) return st;
  ctx->launches += launch_shard_transport(v, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  c.shard_phase = 1;
  return BGK_OK;
}

int bgk_shard_relax(bgk_ctx* ctx, int32_t ci, const double* xm, double* xw, void* stream) {
  CallRange range_("bgk_shard_relax");
  CaseHost* cp = nullptr;
  int st;
  if ((st = shard_case(ctx, ci, xm, false, "bgk_shard_relax", &cp))) return st;
  CaseHost& c = *cp;
  if (!xw && c.cv.n_wall > 0) return fail(ctx, BGK_E_INVAL, "bgk_shard_relax: bad argument");
  if (c.shard_phase != 1) return fail(ctx, BGK_E_STATE, "bgk_shard_relax: call bgk_shard_transport first");
  cudaStream_t s = (cudaStream_t)stream;
  EvPair* e;
  CaseView v = c.cv;
  v.xs = const_cast<double*>(xm);
  if ((st = timed_begin(ctx, K_TRANSPORT, s, &e))) return st;
  ctx->launches += launch_shard_relax(v, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  // the motion reads U^{n+1}, which the relaxation has just stored
  if (c.cv.ale && (st = move_and_prebuild(ctx, c, s))) return st;
  if (c.shard_recon >= 0) CK(ctx, cudaStreamWaitEvent(s, c.ev_recon[c.shard_recon & 1], 0));
  v.xs = xw;
  if ((st = timed_begin(ctx, K_WALLS, s, &e))) return st;
  ctx->launches += launch_shard_walls(v, 1, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  c.shard_phase = 2;
  return BGK_OK;
}

int bgk_shard_walls(bgk_ctx* ctx, int32_t ci, const double* xw, void* stream) {
  CallRange range_("bgk_shard_walls");
  CaseHost* cp = nullptr;
  int st;
  if ((st = shard_case(ctx, ci, xw, true, "bgk_shard_walls", &cp))) return st;
  CaseHost& c = *cp;
  if (c.shard_phase != 2) return fail(ctx, BGK_E_STATE, "bgk_shard_walls: call bgk_shard_relax first");
  cudaStream_t s = (cudaStream_t)stream;
  EvPair* e;
  CaseView v = c.cv;
  v.xs = const_cast<double*>(xw);
  if ((st = timed_begin(ctx, K_WALLS, s, &e))) return st;
  ctx->launches += launch_shard_walls(v, 2, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  c.cur = 1 - c.cur;
  refresh_view(c);
  if (c.next_ready && (st = join_side(ctx, c, s))) return st;
  if ((st = settle_bound(ctx, c, s))) return st;
  c.shard_phase = 0;
  if (ci == 0) ctx->steps += 1;
  return BGK_OK;
}

int bgk_shard_partial(bgk_ctx* ctx, int32_t ci, double* xm, void* stream) {
  CaseHost* cp = nullptr;
  int st;
  if ((st = shard_case(ctx, ci, xm, false, "bgk_shard_partial", &cp))) return st;
  CaseView v = cp->cv;
  v.xs = xm;
  ctx->launches += launch_shard_partial(v, (cudaStream_t)stream);
  CKL(ctx);
  return BGK_OK;
}

int bgk_shard_set_moments(bgk_ctx* ctx, int32_t ci, const double* xm, void* stream) {
  CaseHost* cp = nullptr;
  int st;
  if ((st = shard_case(ctx, ci, xm, false, "bgk_shard_set_moments", &cp))) return st;
  CaseView v = cp->cv;
  v.xs = const_cast<double*>(xm);
  ctx->launches += launch_shard_moments(v, (cudaStream_t)stream);
  CKL(ctx);
  return BGK_OK;
}

int bgk_shard_allreduce(double* const* bufs, int32_t nbufs, int64_t count, void* stream) {
  if (!bufs || nbufs < 1 || nbufs > SHARD_MAX_BUFS || count < 0) return BGK_E_INVAL;
  for (int r = 0; r < nbufs; ++r)
    if (!bufs[r]) return BGK_E_INVAL;
  launch_shard_allreduce(bufs, nbufs, count, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? BGK_OK : BGK_E_CUDA;
}

int bgk_stage_f(bgk_ctx* ctx, int32_t ci, const void* f, int32_t dtype) {
  CallRange range_("bgk_stage_f");
  if (!ctx || !f || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_stage_f: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  if (c.bound || c.slab) return fail(ctx, BGK_E_STATE, "bgk_stage_f: not with bound storage or a velocity slab");
  if (dtype != c.cv.storage || c.cv.NV != c.cv.NVp)
    return fail(ctx, BGK_E_INVAL, "bgk_stage_f: dtype must be the storage type and NV a multiple of 4");
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, f) != cudaSuccess || at.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(ctx, BGK_E_INVAL, "bgk_stage_f: f must be page-locked host memory");
  }
  int st;
  if (!ctx->copy) {
    CK(ctx, cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    for (int k = 0; k < BGK_UPLOAD_PARTS - 1; ++k) {
      CK(ctx, cudaStreamCreateWithFlags(&ctx->copy_part[k], cudaStreamNonBlocking));
      CK(ctx, cudaEventCreateWithFlags(&ctx->ev_part[k], cudaEventDisableTiming));
    }
  }
  if (!c.staged) {
    if ((st = dalloc_bytes(ctx, &c.staged, (size_t)c.cap_n * c.cv.ncomp * c.cv.NVp * c.s_bytes))) return st;
    CK(ctx, cudaEventCreateWithFlags(&c.ev_staged, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&c.ev_free, cudaEventDisableTiming));
  }
  // the staging buffer may be the state buffer a step replaced: wait until that step began
  if (c.free_recorded) CK(ctx, cudaStreamWaitEvent(ctx->copy, c.ev_free, 0));
  // BGK_UPLOAD_PARTS parts of whole rows (one cudaMemcpyAsync each) on as many streams,
  // joined into copy
  const size_t row = (size_t)c.cv.ncomp * c.cv.NVp * c.s_bytes;
  const size_t rows = (size_t)c.cv.n, per = (rows + BGK_UPLOAD_PARTS - 1) / BGK_UPLOAD_PARTS;
  for (int k = 0; k < BGK_UPLOAD_PARTS - 1; ++k) {
    const size_t r0 = std::min(rows, per * (k + 1)), r1 = std::min(rows, per * (k + 2));
    cudaStream_t q = ctx->copy_part[k];
    if (c.free_recorded) CK(ctx, cudaStreamWaitEvent(q, c.ev_free, 0));
    if (r1 > r0)
      CK(ctx, cudaMemcpyAsync(static_cast<char*>(c.staged) + r0 * row, static_cast<const char*>(f) + r0 * row,
                              (r1 - r0) * row, cudaMemcpyHostToDevice, q));
    CK(ctx, cudaEventRecord(ctx->ev_part[k], q));
  }
  CK(ctx, cudaMemcpyAsync(c.staged, f, std::min(rows, per) * row, cudaMemcpyHostToDevice, ctx->copy));
  for (int k = 0; k < BGK_UPLOAD_PARTS - 1; ++k) CK(ctx, cudaStreamWaitEvent(ctx->copy, ctx->ev_part[k], 0));
  CK(ctx, cudaEventRecord(c.ev_staged, ctx->copy));
  c.staged_ready = true;
  return BGK_OK;
}

int bgk_bind_f(bgk_ctx* ctx, int32_t ci, void* f_dev, size_t bytes, void* stream) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_bind_f: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  if (c.staged_ready) return fail(ctx, BGK_E_STATE, "bgk_bind_f: an input staged by bgk_stage_f is pending");
  const size_t rows = (size_t)c.cv.n * c.cv.ncomp * c.cv.NVp * c.s_bytes;
  if (c.bound) {
    // back to the context's own buffer, with the current state in it
    if (c.cur == c.bound_slot) CK(ctx, cudaMemcpyAsync(c.own_buf, c.bound, rows, cudaMemcpyDeviceToDevice, s));
    c.f[c.bound_slot] = c.own_buf;
    c.bound = nullptr;
    c.bound_slot = -1;
    c.own_buf = nullptr;
    refresh_view(c);
    invalidate_batch(ctx);
    CK(ctx, cudaStreamSynchronize(s));
  }
  if (!f_dev) return BGK_OK;
  if (c.cv.NV != c.cv.NVp) return fail(ctx, BGK_E_INVAL, "bgk_bind_f: NV must be a multiple of 4");
  if (reinterpret_cast<uintptr_t>(f_dev) % 16 != 0) return fail(ctx, BGK_E_INVAL, "bgk_bind_f: f_dev must be 16-byte aligned");
  const size_t need = (size_t)c.cap_n * c.cv.ncomp * c.cv.NVp * c.s_bytes;
  if (bytes < need) return fail(ctx, BGK_E_INVAL, "bgk_bind_f: %zu bytes, %zu needed", bytes, need);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, f_dev) != cudaSuccess ||
      (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(ctx, BGK_E_INVAL, "bgk_bind_f: f_dev is not device memory");
  }
  CK(ctx, cudaMemcpyAsync(f_dev, c.f[c.cur], rows, cudaMemcpyDeviceToDevice, s));
  c.own_buf = c.f[c.cur];
  c.f[c.cur] = f_dev;
  c.bound = f_dev;
  c.bound_slot = c.cur;
  refresh_view(c);
  invalidate_batch(ctx);
  return BGK_OK;
}

int bgk_moments(bgk_ctx* ctx, int32_t ci, double* rho, double* u, double* T, int32_t on_device, void* stream) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_moments: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  const size_t n = c.cv.n, sp = sizeof(double) * MOM_STRIDE;
  if (rho) CK(ctx, cudaMemcpy2DAsync(rho, sizeof(double), c.cv.mom, sp, sizeof(double), n, cudaMemcpyDefault, s));
  if (u)
    for (int a = 0; a < c.cv.dim; ++a)
      CK(ctx, cudaMemcpy2DAsync(u + a, sizeof(double) * c.cv.dim, c.cv.mom + 1 + a, sp, sizeof(double), n, cudaMemcpyDefault, s));
  if (T) CK(ctx, cudaMemcpy2DAsync(T, sizeof(double), c.cv.mom + 4, sp, sizeof(double), n, cudaMemcpyDefault, s));
  if (!on_device) CK(ctx, cudaStreamSynchronize(s));
  return BGK_OK;
}

int bgk_get_positions(bgk_ctx* ctx, int32_t ci, double* x, int32_t on_device, void* stream) {
  if (!ctx || !x || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_get_positions: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  CK(ctx, cudaMemcpyAsync(x, c.cv.x, sizeof(double) * c.cv.n * c.cv.dim, cudaMemcpyDefault, s));
  if (!on_device) CK(ctx, cudaStreamSynchronize(s));
  return BGK_OK;
}

int bgk_get_body(bgk_ctx* ctx, int32_t ci, double* centre) {
  if (!ctx || !centre || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_get_body: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  if (!c.cv.body) return fail(ctx, BGK_E_INVAL, "bgk_get_body: case %d has no body", ci);
  CK(ctx, cudaDeviceSynchronize());
  CK(ctx, cudaMemcpy(centre, reinterpret_cast<const double*>(c.cv.body), sizeof(double) * c.cv.dim, cudaMemcpyDeviceToHost));
  return BGK_OK;
}

int bgk_sync(bgk_ctx* ctx, void* stream) {
  if (!ctx) return BGK_E_INVAL;
  CK(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  CK(ctx, cudaGetLastError());
  DevStatus hs;
  CK(ctx, cudaMemcpy(&hs, ctx->status, sizeof(hs), cudaMemcpyDeviceToHost));
  if (hs.flags) {
    CK(ctx, cudaMemset(&ctx->status->flags, 0, sizeof(int32_t)));
    if (hs.flags & ST_TIMEOUT) {
      // a grid barrier of the side chain gave up: the CTAs that waited left the kernel,
      // so its barrier counter and the lists it was building are incomplete.  Reset the
      // barrier state (and force a candidate rebuild) and discard those lists: the next
      // step builds its lists from the current positions, which the motion phase (before
      // the first barrier) finished.
      for (auto& c : ctx->cases) {
        if (int st = reset_skin(ctx, c)) return st;
        c.next_ready = false;
      }
    }
    // the first condition in this order (bounds, overflow, singular, non-finite, timeout)
    // is the return code; the text names every one
    char all[96];
    snprintf(all, sizeof(all), " (device flags:%s%s%s%s%s)", hs.flags & ST_BOUNDS ? " bounds" : "",
             hs.flags & ST_OVERFLOW ? " overflow" : "", hs.flags & ST_SINGULAR ? " singular" : "",
             hs.flags & ST_NONFINITE ? " nonfinite" : "", hs.flags & ST_TIMEOUT ? " timeout" : "");
    if (hs.flags & ST_BOUNDS)
      return fail(ctx, BGK_E_BOUNDS, "an index outside the point range was found and skipped%s", all);
    if (hs.flags & ST_OVERFLOW) return fail(ctx, BGK_E_NBR_OVERFLOW, "a point has more than max_nbrs neighbours%s", all);
    if (hs.flags & ST_SINGULAR)
      return fail(ctx, BGK_E_SINGULAR, "singular WLS system (too few or degenerate neighbours)%s", all);
    if (hs.flags & ST_NONFINITE)
      return fail(ctx, BGK_E_NONFINITE, "non-finite or non-positive density or temperature%s", all);
    if (hs.flags & ST_TIMEOUT) return fail(ctx, BGK_E_TIMEOUT, "a bounded device wait gave up%s", all);
  }
  return BGK_OK;
}

static const uint64_t kMagic = 0x31544154534b4742ull;  // "BGKSTAT1"

int bgk_get_state(bgk_ctx* ctx, void* blob, size_t cap, size_t* used) {
  if (!ctx || !used) return BGK_E_INVAL;
  size_t need = 4 * sizeof(uint64_t);
  for (auto& c : ctx->cases)
    need += 4 * sizeof(int64_t) + sizeof(double) * c.cv.n * c.cv.dim +
            (size_t)c.cv.n * c.cv.ncomp * c.cv.NVp * c.s_bytes + sizeof(double) * c.cv.n * MOM_STRIDE +
            sizeof(double) * 3;
  *used = need;
  if (!blob) return BGK_OK;
  if (cap < need) return fail(ctx, BGK_E_INVAL, "bgk_get_state: cap %zu < %zu", cap, need);
  CK(ctx, cudaDeviceSynchronize());
  unsigned char* o = static_cast<unsigned char*>(blob);
  uint64_t hdr[4] = {kMagic, (uint64_t)BGK_ABI_VERSION, (uint64_t)ctx->cases.size(), (uint64_t)ctx->steps};
  memcpy(o, hdr, sizeof(hdr));
  o += sizeof(hdr);
  for (auto& c : ctx->cases) {
    int64_t ch[4] = {c.cv.n, c.cv.dim, c.cv.NVp, c.p.storage};
    memcpy(o, ch, sizeof(ch));
    o += sizeof(ch);
    size_t b = sizeof(double) * c.cv.n * c.cv.dim;
    CK(ctx, cudaMemcpy(o, c.cv.x, b, cudaMemcpyDeviceToHost));
    o += b;
    b = (size_t)c.cv.n * c.cv.ncomp * c.cv.NVp * c.s_bytes;
    CK(ctx, cudaMemcpy(o, c.f[c.cur], b, cudaMemcpyDeviceToHost));
    o += b;
    b = sizeof(double) * c.cv.n * MOM_STRIDE;
    CK(ctx, cudaMemcpy(o, c.cv.mom, b, cudaMemcpyDeviceToHost));
    o += b;
    double bc[3] = {0.0, 0.0, 0.0};
    if (c.cv.body) CK(ctx, cudaMemcpy(bc, reinterpret_cast<const double*>(c.cv.body), sizeof(bc), cudaMemcpyDeviceToHost));
    memcpy(o, bc, sizeof(bc));
    o += sizeof(bc);
  }
  return BGK_OK;
}

int bgk_set_state(bgk_ctx* ctx, const void* blob, size_t size) {
  if (!ctx || !blob) return BGK_E_INVAL;
  size_t need = 0;
  bgk_get_state(ctx, nullptr, 0, &need);
  if (size != need) return fail(ctx, BGK_E_STATE, "bgk_set_state: blob size %zu != %zu", size, need);
  const unsigned char* o = static_cast<const unsigned char*>(blob);
  uint64_t hdr[4];
  memcpy(hdr, o, sizeof(hdr));
  o += sizeof(hdr);
  if (hdr[0] != kMagic || hdr[1] != (uint64_t)BGK_ABI_VERSION || hdr[2] != ctx->cases.size())
    return fail(ctx, BGK_E_STATE, "bgk_set_state: blob does not match this context");
  CK(ctx, cudaDeviceSynchronize());
  for (auto& c : ctx->cases) {
    int64_t ch[4];
    memcpy(ch, o, sizeof(ch));
    o += sizeof(ch);
    if (ch[0] != c.cv.n || ch[1] != c.cv.dim || ch[2] != c.cv.NVp || ch[3] != c.p.storage)
      return fail(ctx, BGK_E_STATE, "bgk_set_state: case layout mismatch");
    size_t b = sizeof(double) * c.cv.n * c.cv.dim;
    CK(ctx, cudaMemcpy(c.cv.x, o, b, cudaMemcpyHostToDevice));
    o += b;
    b = (size_t)c.cv.n * c.cv.ncomp * c.cv.NVp * c.s_bytes;
    CK(ctx, cudaMemcpy(c.f[0], o, b, cudaMemcpyHostToDevice));
    o += b;
    b = sizeof(double) * c.cv.n * MOM_STRIDE;
    CK(ctx, cudaMemcpy(c.cv.mom, o, b, cudaMemcpyHostToDevice));
    o += b;
    if (c.cv.body) {
      BodyState b0;
      memset(&b0, 0, sizeof(b0));
      memcpy(b0.c, o, sizeof(b0.c));
      CK(ctx, cudaMemcpy(c.cv.body, &b0, sizeof(b0), cudaMemcpyHostToDevice));
    }
    o += 3 * sizeof(double);
    c.stencils_valid = false;
    c.shard_phase = 0;
    c.staged_ready = false;
    if (int st = reset_skin(ctx, c)) return st;  // positions changed: rebuild the candidates
    c.cur = 0;
    refresh_view(c);
    if (int st = settle_bound(ctx, c, 0)) return st;
  }
  CK(ctx, cudaDeviceSynchronize());
  invalidate_batch(ctx);
  ctx->steps = (int64_t)hdr[3];
  return BGK_OK;
}

int bgk_set_params(bgk_ctx* ctx, int32_t ci, const bgk_params* p) {
  if (!ctx || !p || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_set_params: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  const bgk_params& o = c.p;
  const char* why = nullptr;
  if (!check_params(*p, c.cv.n, &why)) return fail(ctx, BGK_E_INVAL, "bgk_set_params: %s", why);
  if (p->dim != o.dim || p->nv != o.nv || p->vmax != o.vmax || p->storage != o.storage || p->max_nbrs != o.max_nbrs ||
      p->h != o.h || p->alpha != o.alpha || p->periodic != o.periodic || p->skin != o.skin ||
      p->spare_points != o.spare_points || p->wls_order != o.wls_order || p->body_wall != o.body_wall ||
      p->vk_lo != o.vk_lo || p->vk_hi != o.vk_hi || p->time_order != o.time_order || p->vgrid != o.vgrid ||
      p->body_radius != o.body_radius ||
      p->body_centre[0] != o.body_centre[0] || p->body_centre[1] != o.body_centre[1] ||
      p->body_centre[2] != o.body_centre[2])
    return fail(ctx, BGK_E_INVAL,
                "bgk_set_params: only kn, tau_mode, dt, wall_T, lid_u, lid_wall, ale, guard, body_u may change");
  CK(ctx, cudaDeviceSynchronize());
  c.p = *p;
  CaseView& v = c.cv;
  v.kn = p->kn;
  v.tau_mode = p->tau_mode;
  v.dt = p->dt;
  set_case_consts(v);
  v.wall_T = p->wall_T;
  v.lid_wall = p->lid_wall;
  if (v.ale != p->ale) {
    // the points may have moved since the lists were built: rebuild them at the next step
    int st = reset_skin(ctx, c);
    if (st) return st;
    c.stencils_valid = false;
  }
  v.ale = p->ale;
  v.guard = p->guard;
  for (int a = 0; a < 3; ++a) v.lid_u[a] = p->lid_u[a];
  for (int a = 0; a < 3; ++a) v.body_u[a] = p->body_u[a];
  v.body_rg = p->body_radius + p->guard;
  refresh_view(c);
  ctx->launches += launch_init_tables(v, 0);
  CKL(ctx);
  CK(ctx, cudaDeviceSynchronize());
  invalidate_batch(ctx);
  return BGK_OK;
}

int bgk_manage(bgk_ctx* ctx, int32_t ci, double rmin, int32_t min_nbrs, int64_t* counts, void* stream) {
  CallRange range_("bgk_manage");
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || !counts || !(rmin >= 0) || min_nbrs < 0)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_manage: bad argument") : BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CaseHost& c = ctx->cases[ci];
  if (c.slab) return fail(ctx, BGK_E_STATE, "bgk_manage: not available for a velocity slab");
  c.staged_ready = false;  // a pending staged input has the old point count: dropped
  int st;
  if ((st = join_side(ctx, c, s))) return st;
  refresh_view(c);
  const int dim = c.cv.dim;
  const size_t cn = c.cap_n;
  if (!c.pm_nn) {
    if ((st = dalloc(ctx, &c.pm_nn, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_role, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_newidx, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_addidx, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_totals, 2))) return st;
    if ((st = dalloc(ctx, &c.pm_kind2, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_int2, cn))) return st;
    if ((st = dalloc(ctx, &c.pm_ynew, cn * dim))) return st;
    if ((st = dalloc(ctx, &c.pm_x2, cn * dim))) return st;
    if ((st = dalloc(ctx, &c.pm_norm2, cn * dim))) return st;
  }
  // exact lists of the current positions
  CaseView v = c.cv;
  ctx->launches += launch_neighbours(v, s);
  // the skin path expects zero cell counts at the start of a rebuild
  if (v.sk) CK(ctx, cudaMemsetAsync(v.cell_cnt, 0, sizeof(int32_t) * v.ncell, s));
  ctx->launches += launch_manage_plan(v, rmin, min_nbrs, c.pm_nn, c.pm_role, c.pm_ynew, c.pm_newidx, c.pm_addidx,
                                      c.pm_totals, s);
  CKL(ctx);
  int32_t tot[2];
  CK(ctx, cudaMemcpyAsync(tot, c.pm_totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  const int64_t n_old = v.n, survivors = tot[0];
  const int64_t adds = std::min<int64_t>(tot[1], c.cap_n - survivors);
  const int64_t n_new = survivors + adds;
  ctx->launches += launch_manage_apply(v, c.cap_n, c.pm_nn, c.pm_role, c.pm_ynew, c.pm_newidx, c.pm_addidx,
                                       c.pm_totals, c.pm_x2, c.pm_kind2, c.pm_norm2, c.f[c.cur], c.f[1 - c.cur],
                                       c.pm_int2, const_cast<int32_t*>(c.cv.wall_idx), c.wall_of, n_new, s);
  CKL(ctx);
  // the new arrays become current
  {
    double* t = c.cv.x; c.cv.x = c.pm_x2; c.pm_x2 = t;
  }
  {
    int32_t* t = const_cast<int32_t*>(c.cv.kind); c.cv.kind = c.pm_kind2; c.pm_kind2 = t;
  }
  {
    double* t = const_cast<double*>(c.cv.normal); c.cv.normal = c.pm_norm2; c.pm_norm2 = t;
  }
  {
    int32_t* t = const_cast<int32_t*>(c.cv.int_idx); c.cv.int_idx = c.pm_int2; c.pm_int2 = t;
  }
  c.cur = 1 - c.cur;
  c.cv.n_int = (int32_t)(c.cv.n_int - (n_old - survivors) + adds);
  c.cv.n = (int32_t)n_new;
  refresh_view(c);
  ctx->launches += launch_moments(c.cv, c.f[c.cur], s);
  CKL(ctx);
  CK(ctx, cudaStreamSynchronize(s));
  c.stencils_valid = false;
  c.next_ready = false;
  c.tslot_valid = false;
  if ((st = reset_skin(ctx, c))) return st;
  invalidate_batch(ctx);
  if ((st = settle_bound(ctx, c, s))) return st;
  CK(ctx, cudaStreamSynchronize(s));
  counts[0] = n_new;
  counts[1] = n_old - survivors;
  counts[2] = adds;
  return BGK_OK;
}

int bgk_objective(bgk_ctx* ctx, int32_t ci, double* J, void* lam, double scale, void* stream) {
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size())
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_objective: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  if (c.slab) return fail(ctx, BGK_E_STATE, "bgk_objective: not available for a velocity slab");
  refresh_view(c);
  ctx->launches += launch_objective(c.cv, c.nlid, J, lam, scale, (cudaStream_t)stream);
  CKL(ctx);
  return BGK_OK;
}

int bgk_adjoint_step(bgk_ctx* ctx, int32_t ci, const void* lam_in, void* lam_out, double* dtheta, void* stream) {
  CallRange range_("bgk_adjoint_step");
  if (!ctx || ci < 0 || ci >= (int)ctx->cases.size() || !lam_in || !lam_out || !dtheta || lam_in == lam_out)
    return ctx ? fail(ctx, BGK_E_INVAL, "bgk_adjoint_step: bad argument") : BGK_E_INVAL;
  CaseHost& c = ctx->cases[ci];
  if (c.cv.ale) return fail(ctx, BGK_E_STATE, "bgk_adjoint_step: the adjoint is for fixed points (ale = 0)");
  if (c.slab) return fail(ctx, BGK_E_STATE, "bgk_adjoint_step: not available for a velocity slab");
  if (c.p.time_order == 2) return fail(ctx, BGK_E_STATE, "bgk_adjoint_step: the adjoint is of the first-order step");
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  refresh_view(c);
  if (!c.stencils_valid && (st = build_lists(ctx, c, s))) return st;
  const size_t fl = (size_t)c.cap_n * c.cv.ncomp * c.cv.NVp * c.c_bytes;
  if (!c.adj_ft) {
    if ((st = dalloc_bytes(ctx, &c.adj_ft, fl))) return st;
    if ((st = dalloc_bytes(ctx, &c.adj_y, fl))) return st;
    if ((st = dalloc_bytes(ctx, &c.adj_lft, fl))) return st;
    if ((st = dalloc(ctx, &c.adj_wmu, std::max<int64_t>(c.cv.n_wall, 1)))) return st;
    if ((st = dalloc(ctx, &c.adj_mom, (size_t)c.cap_n * MOM_STRIDE))) return st;
    if ((st = dalloc(ctx, &c.adj_sk, (size_t)c.cap_n * c.cv.NVp))) return st;
    if ((st = dalloc(ctx, &c.tslot, (size_t)c.cap_n * c.cv.cap))) return st;
    CK(ctx, cudaMemset(c.adj_lft, 0, fl));
  }
  if (!c.tslot_valid) {
    ctx->launches += launch_tslot(c.cv, c.tslot, s);
    CKL(ctx);
    c.tslot_valid = true;
  }
  EvPair* e;
  if ((st = timed_begin(ctx, K_ADJOINT, s, &e))) return st;
  if (c.cv.storage != 1)  // FP64 and BF16 storage: generic kernels; FP32 storage: warp-per-point kernels
    ctx->launches += launch_adjoint(c.cv, lam_in, lam_out, dtheta, c.adj_ft, c.adj_y, c.adj_lft, c.adj_wmu, c.tslot,
                                    c.wall_of, s);
  else
    ctx->launches += launch_adjoint_fp32(c.cv, lam_in, lam_out, dtheta, c.adj_ft, c.adj_y, c.adj_lft, c.adj_wmu,
                                         c.adj_mom, c.adj_sk, c.tslot, c.wall_of, s);
  CKL(ctx);
  if ((st = timed_end(ctx, e, s))) return st;
  return BGK_OK;
}

int bgk_set_batching(bgk_ctx* ctx, int32_t mode) {
  if (!ctx || mode < -1 || mode > 2) return ctx ? fail(ctx, BGK_E_INVAL, "bgk_set_batching: mode in -1..2") : BGK_E_INVAL;
  ctx->batch_mode = mode;
  drop_graphs(ctx);
  return BGK_OK;
}

int bgk_autotune(bgk_ctx* ctx, void* stream) {
  if (!ctx) return BGK_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!batch_eligible(ctx)) return BGK_OK;  // nothing to tune: per-case launches
  int st;
  if ((st = prepare_batch(ctx, s))) return st;
  int dev = 0, nsm = 0;
  CK(ctx, cudaGetDevice(&dev));
  CK(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int parity = ctx->cases[0].cur;
  cudaEvent_t e0, e1;
  CK(ctx, cudaEventCreate(&e0));
  CK(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int bw = ctx->batch_warps, bg = ctx->batch_grid;
  const int warps_c[2] = {4, 8};
  const int mult_c[6] = {0, 1, 2, 3, 4, 6};
  for (int wi = 0; wi < 2; ++wi)
    for (int mi = 0; mi < 6; ++mi) {
      const int grid = mult_c[mi] * nsm;
      // the transport launch reads f_in and writes f_out only, so repeating it leaves the state unchanged
      for (int rep = 0; rep < 6; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        ctx->launches += launch_transport_batch(ctx->d_cases[parity], ctx->d_items, ctx->n_items, ctx->batch_dim,
                                                ctx->batch_storage, ctx->capmax, warps_c[wi], grid, s);
      }
      cudaEventRecord(e1, s);
      CKL(ctx);
      CK(ctx, cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bw = warps_c[wi]; bg = grid; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->batch_warps = bw;
  ctx->batch_grid = bg;
  drop_graphs(ctx);
  return BGK_OK;
}

int bgk_set_watchdog(bgk_ctx* ctx, int64_t max_polls) {
  if (!ctx || max_polls < 0) return ctx ? fail(ctx, BGK_E_INVAL, "bgk_set_watchdog: max_polls < 0") : BGK_E_INVAL;
  ctx->watchdog = max_polls;
  return BGK_OK;
}

int bgk_set_timing(bgk_ctx* ctx, int32_t enable) {
  if (!ctx) return BGK_E_INVAL;
  int st = collect_timing(ctx);
  if (st) return st;
  ctx->timing_mask = enable;
  ctx->timing = enable != 0;
  // pre-create event pairs so that timed regions do not pay for cudaEventCreate
  while (ctx->timing && ctx->ev.size() < 8192) {
    EvPair e;
    CK(ctx, cudaEventCreate(&e.a));
    CK(ctx, cudaEventCreate(&e.b));
    e.kid = 0;
    ctx->ev.push_back(e);
  }
  for (int k = 0; k < K_COUNT; ++k) { ctx->t_ms[k] = 0.0; ctx->t_n[k] = 0; }
  return BGK_OK;
}

int bgk_get_timing(bgk_ctx* ctx, int32_t which, double* total_ms, int64_t* launches) {
  if (!ctx || which < 0 || which >= K_COUNT || !total_ms || !launches) return BGK_E_INVAL;
  int st = collect_timing(ctx);
  if (st) return st;
  *total_ms = ctx->t_ms[which];
  *launches = ctx->t_n[which];
  return BGK_OK;
}

int bgk_get_stats(bgk_ctx* ctx, bgk_stats* out) {
  if (!ctx || !out) return BGK_E_INVAL;
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  cudaMemcpy(&hs, ctx->status, sizeof(hs), cudaMemcpyDeviceToHost);
  out->steps = ctx->steps;
  out->launches = ctx->launches;
  out->clamps = (int64_t)hs.clamps;
  out->nnz = 0;
  for (auto& c : ctx->cases) {
    std::vector<int32_t> cnt(c.cv.n);
    cudaMemcpy(cnt.data(), c.cv.cnt, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost);
    for (int32_t v : cnt) out->nnz += v;
  }
  out->nv_pad = ctx->cases.empty() ? 0 : ctx->cases[0].cv.NVp;
  out->n_cases = (int32_t)ctx->cases.size();
  out->batch_mode = effective_mode(ctx);
  out->batch_warps = ctx->batch_warps;
  out->batch_grid = ctx->batch_grid;
  return BGK_OK;
}

const char* bgk_last_error(const bgk_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

void bgk_free(bgk_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  drop_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->copy) cudaStreamDestroy(ctx->copy);
  for (int k = 0; k < BGK_UPLOAD_PARTS - 1; ++k) {
    if (ctx->copy_part[k]) cudaStreamDestroy(ctx->copy_part[k]);
    if (ctx->ev_part[k]) cudaEventDestroy(ctx->ev_part[k]);
  }
  for (auto& c : ctx->cases) {
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_staged) cudaEventDestroy(c.ev_staged);
    if (c.ev_free) cudaEventDestroy(c.ev_free);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    for (int k = 0; k < 2; ++k)
      if (c.ev_recon[k]) cudaEventDestroy(c.ev_recon[k]);
  }
  for (auto& e : ctx->ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->staging) cudaFree(ctx->staging);
  delete ctx;
}

}  // extern "C"
