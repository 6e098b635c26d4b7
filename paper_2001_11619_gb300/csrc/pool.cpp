// Process-wide cache of device allocations.
//
// A factorization allocates its factor arenas, the bordered columns
// (2N x 3p doubles each: 12.9 GB apiece on the 1M-node, 256-hole case) and
// per-level scratch.  cudaMalloc and cudaFree of such sizes cost
// milliseconds to seconds (pages are mapped and unmapped, and cudaFree
// synchronises the device), and a program that builds many solvers (a
// shape-optimisation loop, a benchmark, the hole-move trials of the
// replica driver) would pay that each time.  Freed blocks are therefore
// kept per device and handed out again for requests of at most their size
// and at least half of it.  The cache holds at most half of the device's
// memory (SKEL_CACHE_LIMIT_GB overrides; 0 turns caching off), and
// skel_release_cached_memory returns every cached block to the driver.
// A failed cudaMalloc releases the cache and tries once more.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdlib>
#include <map>
#include <mutex>
#include <unordered_map>

#include "skel_internal.h"

namespace skel {

namespace {

struct Block {
  size_t bytes;
  int dev;
};

std::mutex g_mu;
std::unordered_map<void *, Block> g_live;          // handed out
std::map<int, std::multimap<size_t, void *>> g_free;  // per device, by size
size_t g_cached = 0;
long long g_limit = -1;  // bytes; -1: not yet read
std::atomic<long long> g_alloc_ns{0};

size_t round_up(size_t b) {
  const size_t g = b >= ((size_t)1 << 20) ? ((size_t)2 << 20) : 512;
  return (b + g - 1) / g * g;
}

long long limit_bytes() {
  if (g_limit >= 0) return g_limit;
  const char *e = std::getenv("SKEL_CACHE_LIMIT_GB");
  if (e && *e) {
    g_limit = (long long)(std::atof(e) * 1e9);
  } else {
    size_t fr = 0, tot = 0;
    g_limit = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? (long long)(tot / 2)
                                                        : 0;
  }
  if (g_limit < 0) g_limit = 0;
  return g_limit;
}

struct Clock {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  ~Clock() {
    g_alloc_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(
                      std::chrono::steady_clock::now() - t0)
                      .count();
  }
};

// cudaFree every cached block (caller holds g_mu)
void release_locked() {
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto &kv : g_free) {
    if (kv.second.empty()) continue;
    cudaSetDevice(kv.first);
    for (auto &b : kv.second) cudaFree(b.second);
    kv.second.clear();
  }
  cudaSetDevice(cur);
  g_cached = 0;
}

}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes) {
  Clock clk;
  *p = nullptr;
  const size_t want = round_up(bytes == 0 ? 1 : bytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  auto &fl = g_free[dev];
  auto it = fl.lower_bound(want);
  if (it != fl.end() && it->first <= 2 * want) {
    *p = it->second;
    g_live[*p] = Block{it->first, dev};
    g_cached -= it->first;
    fl.erase(it);
    return cudaSuccess;
  }
  e = cudaMalloc(p, want);
  if (e == cudaErrorMemoryAllocation && g_cached > 0) {
    (void)cudaGetLastError();
    release_locked();
    e = cudaMalloc(p, want);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_live[*p] = Block{want, dev};
  return cudaSuccess;
}

void dev_free(void *p) {
  if (!p) return;
  Clock clk;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) {  // not from dev_alloc
    cudaFree(p);
    return;
  }
  const Block b = it->second;
  g_live.erase(it);
  if ((long long)(g_cached + b.bytes) <= limit_bytes()) {
    g_free[b.dev].emplace(b.bytes, p);
    g_cached += b.bytes;
    return;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b.dev) cudaSetDevice(b.dev);
  cudaFree(p);
  if (cur != b.dev) cudaSetDevice(cur);
}

double dev_alloc_ms() { return g_alloc_ns.load() * 1e-6; }

size_t dev_cached_bytes() {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_cached;
}

}  // namespace skel

extern "C" int skel_release_cached_memory(void) {
  std::lock_guard<std::mutex> lock(skel::g_mu);
  skel::release_locked();
  return cudaGetLastError() == cudaSuccess ? SKEL_OK : SKEL_ECUDA;
}
