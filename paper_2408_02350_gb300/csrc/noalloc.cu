// bgk_neighbours_noalloc: the neighbour-list build for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a memory manager
// which owns the whole device heap (a caching allocator that must see every
// allocation), or code that is not allowed to allocate once it has started
// (fixed memory budgets, long-running services).  For them this entry point
// builds the neighbour lists into buffers the caller already owns and keeps its
// scratch (cell lists, an FP32 copy of the positions, a status word) in one
// fixed-size array in device global memory that is part of the library image.
//
// The array exists once per GPU that loads the library and stays resident
// until the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it; make that
// first call before any stream capture.  All calls share the array: the
// scratch that must start at zero (cell counters, status word) is cleared at
// the start of every call, and calls whose work overlaps on the GPU (different
// streams without ordering) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "bgk.h"
#include "bgk_internal.cuh"

namespace bgk {
namespace {

constexpr int64_t kMaxPoints = 131072;  // BGK_NOALLOC_MAX_POINTS
constexpr int64_t kMaxCells = 131072;   // BGK_NOALLOC_MAX_CELLS
constexpr int kMaxDevices = 64;

constexpr size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffCellOf = 256;
constexpr size_t kOffCellPts = kOffCellOf + round256(4 * kMaxPoints);
constexpr size_t kOffXf = kOffCellPts + round256(4 * kMaxPoints);
constexpr size_t kOffCellStart = kOffXf + round256(4 * 3 * kMaxPoints);
constexpr size_t kOffCellCnt = kOffCellStart + round256(4 * (kMaxCells + 1));
constexpr size_t kScratchBytes = kOffCellCnt + round256(4 * kMaxCells);  // about 3.7 MB
static_assert(sizeof(DevStatus) <= 256, "status slot");

static __device__ __align__(256) unsigned char g_nbr_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of g_nbr_scratch on the current device (looked up once per device).
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return BGK_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_nbr_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BGK_E_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch[dev]);
  return BGK_OK;
}

}  // namespace
}  // namespace bgk

extern "C" int bgk_neighbours_noalloc(int32_t dim, int64_t n, const double* x, double h, int32_t periodic,
                                      int32_t cap, int32_t* cnt, int32_t* col, int32_t check, void* stream) {
  using namespace bgk;
  if ((dim != 2 && dim != 3) || n < 1 || n > kMaxPoints || !(h > 0.0) || cap < 1 || cap > 443 || !x || !cnt ||
      !col)
    return BGK_E_INVAL;
  int nc = (int)std::floor(1.0 / (h * (1.0 + 1e-9)));
  if (nc < 1) nc = 1;
  int64_t ncell = 1;
  for (int a = 0; a < dim; ++a) ncell *= nc;
  if (ncell > kMaxCells) return BGK_E_INVAL;
  unsigned char* base = nullptr;
  int st = scratch_address(&base);
  if (st != BGK_OK) return st;

  CaseView cv;
  memset(&cv, 0, sizeof(cv));
  cv.dim = dim;
  cv.n = (int32_t)n;
  cv.cap = cap;
  cv.periodic = periodic;
  cv.h = h;
  set_case_consts(cv);  // h^2 for the exact neighbour test
  cv.nc = nc;
  cv.ncell = (int32_t)ncell;
  cv.x = const_cast<double*>(x);
  cv.cnt = cnt;
  cv.col = col;
  cv.status = reinterpret_cast<DevStatus*>(base + kOffStatus);
  cv.cell_of = reinterpret_cast<int32_t*>(base + kOffCellOf);
  cv.cell_pts = reinterpret_cast<int32_t*>(base + kOffCellPts);
  cv.xf = reinterpret_cast<float*>(base + kOffXf);
  cv.cell_start = reinterpret_cast<int32_t*>(base + kOffCellStart);
  cv.cell_cnt = reinterpret_cast<int32_t*>(base + kOffCellCnt);

  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(cv.status, 0, sizeof(DevStatus), s) != cudaSuccess) {
    cudaGetLastError();
    return BGK_E_CUDA;
  }
  launch_neighbours(cv, s);  // clears the cell counters itself
  if (cudaGetLastError() != cudaSuccess) return BGK_E_CUDA;
  if (check) {
    DevStatus hs;
    if (cudaMemcpyAsync(&hs, cv.status, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return BGK_E_CUDA;
    }
    if (hs.flags & ST_OVERFLOW) return BGK_E_NBR_OVERFLOW;
  }
  return BGK_OK;
}
