// Scratch for skel_eval_velocity_noalloc: the partial sums of the velocity
// evaluation live in one fixed device array, defined here, instead of memory
// allocated at run time.  The array is shared by every call in the process;
// calls that overlap on the GPU race on it.
#include <cuda.h>  // CUcontext and CUresult (types only; no driver link)

#include <mutex>

#include "skel_internal.h"

namespace skel {

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
// The array's device address per device, valid for the context that was
// current when it was looked up (by the context's id, which the driver
// never reuses within a process).  After a device reset or with another
// context the address is looked up again.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  double *addr = nullptr;
};
ScratchAddr g_noalloc_addr[kMaxDevices];

// two driver calls, resolved through the runtime (no link to libcuda)
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
void *driver_fn(const char *name) {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

// id of the context current on this thread, or 0 if there is none
bool current_ctx_id(unsigned long long *id) {
  static CtxGetCurrentFn get_cur =
      reinterpret_cast<CtxGetCurrentFn>(driver_fn("cuCtxGetCurrent"));
  static CtxGetIdFn get_id =
      reinterpret_cast<CtxGetIdFn>(driver_fn("cuCtxGetId"));
  if (!get_cur || !get_id) return false;
  CUcontext cur = nullptr;
  *id = 0;
  if (get_cur(&cur) != CUDA_SUCCESS || !cur) return true;
  return get_id(cur, id) == CUDA_SUCCESS;
}
}  // namespace

// Set-up, once per device and context, with that device current: look up
// the array's device address.  Later calls in the same context reuse it;
// a call in another context (after a device reset, say) looks it up anew.
static int noalloc_scratch(double **ptr, std::string &err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return SKEL_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal beyond the static scratch table";
    return SKEL_EINVAL;
  }
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) {
    err = "cuCtxGetCurrent / cuCtxGetId are not available from the driver";
    return SKEL_ECUDA;
  }
  if (id == 0) {
    // no context yet on this thread: the runtime makes the device's
    // primary context current on its first call that needs one
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !current_ctx_id(&id) || id == 0) {
      err = "no CUDA context on the current device";
      return SKEL_ECUDA;
    }
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  ScratchAddr &slot = g_noalloc_addr[dev];
  if (!slot.addr || slot.ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return SKEL_ECUDA;
    }
    slot.addr = static_cast<double *>(p);
    slot.ctx_id = id;
  }
  *ptr = slot.addr;
  return SKEL_OK;
}

int launch_eval_velocity_noalloc(const DevGeom &g, int nrhs, const double *sol,
                                 int64_t ld, int64_t nt, const double *tx,
                                 const double *ty, double *u, cudaStream_t s,
                                 std::string &err) {
  double *scratch = nullptr;
  const int rc = noalloc_scratch(&scratch, err);
  if (rc != SKEL_OK) return rc;
  // The first kernel writes every partial sum that the second one reads, so
  // nothing in the array has to start at zero.
  if (!launch_eval_velocity_capped(g, nrhs, sol, ld, nt, tx, ty, u, scratch,
                                   kNoallocScratchDoubles, s)) {
    err = "nt * nrhs exceeds the static scratch";
    return SKEL_ECAPACITY;
  }
  return SKEL_OK;
}

}  // namespace skel
