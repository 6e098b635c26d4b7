// Scratch for skel_eval_velocity_noalloc: the partial sums of the velocity
// evaluation live in one fixed device array, defined here, instead of memory
// allocated at run time.  The array is shared by every call in the process;
// calls that overlap on the GPU race on it.
#include <mutex>

#include "skel_internal.h"

namespace skel {

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// Set-up, once per device with that device current: look up the array's
// device address.  Later calls on the same device reuse it.
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
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return SKEL_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *ptr = g_noalloc_addr[dev];
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
