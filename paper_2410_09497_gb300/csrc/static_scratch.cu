// A variant of the patch smoother that allocates no device memory.
//
// stk_smooth keeps its per-colour residual in workspace that the library
// allocates with cudaMalloc on first use.  Some callers cannot allow that: a
// framework that owns every device allocation through its own pool and
// forbids others (a foreign cudaMalloc would escape its accounting and could
// fail once the pool has taken the memory), or a real-time host loop where a
// cudaMalloc, which may synchronise the device, is an unacceptable stall.
// stk_smooth_static
// runs the same kernels in the same order, with the residual held in one
// fixed array in device global memory that is part of the library image.
//
// The array holds kStaticScratchBytes (32 MiB): up to 4,194,304 FP64 or
// 8,388,608 FP32 entries, i.e. levels with N at most that (16^3 cells at
// k = 5, 32^3 cells at k = 2 in FP64).  Every GPU that loads the library
// reserves it until the process exits.  Calls share it: the residual of the
// last call stays there, and two calls that overlap on the GPU (different
// streams, or different problems without ordering between them) race on it.
#include <mutex>

#include "internal.h"

namespace stk {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;

// The residual of the current colour.  The residual kernel overwrites every
// entry of the level it is called for (constrained rows are written as 0), so
// nothing has to be cleared between calls.
static __device__ __align__(256) unsigned char g_smooth_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_smooth_scratch on the current device.  In host code the
// symbol name is only a host-side handle, so the address is looked up once
// per device with cudaGetSymbolAddress (the device must be current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_smooth_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace stk

extern "C" int stk_smooth_static(stk_problem* P, int level, int dtype, void* x, const void* b) {
  if (!P) return STK_EINVAL;
  if (P->dim != 3) {
    P->err = "smooth_static: three-dimensional problems only";
    return STK_EINVAL;
  }
  if (level < 0 || level >= (int)P->levels.size()) {
    P->err = "level out of range";
    return STK_EINVAL;
  }
  if (dtype != STK_F64 && dtype != STK_F32) {
    P->err = "dtype must be STK_F64 or STK_F32";
    return STK_EINVAL;
  }
  if (!x || !b || (reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u)) {
    P->err = "x and b must be non-NULL and 16-byte aligned";
    return STK_EINVAL;
  }
  if (x == b) {
    P->err = "x and b must not alias";
    return STK_EINVAL;
  }
  const size_t need = (size_t)P->levels[level].ntotal * (dtype == STK_F64 ? 8 : 4);
  if (need > stk::kStaticScratchBytes) {
    P->err = "level too large for stk_smooth_static: needs " + std::to_string(need) +
             " bytes of residual scratch, the static array holds " + std::to_string(stk::kStaticScratchBytes);
    return STK_EINVAL;
  }
  if (P->opt.local_cg_mode == STK_LOCAL_DIRECT && !P->levels[level].dir_ready) {
    // building the Direct local inverses allocates: a stk_smooth call on the level does it
    P->err = "smooth_static: the Direct local inverses of this level are not built yet";
    return STK_ESTATE;
  }
  void* r = nullptr;
  cudaError_t e = stk::scratch_address(&r);
  for (int colour = 0; e == cudaSuccess && colour < 8; ++colour) {
    e = stk::launch_apply(P, level, dtype, x, b, r, -1.0);
    if (e == cudaSuccess) e = stk::launch_patch_colour(P, level, dtype, colour, r, x);
  }
  if (e != cudaSuccess) {
    P->err = std::string("smooth_static: ") + cudaGetErrorString(e);
    return STK_ECUDA;
  }
  return STK_OK;
}
