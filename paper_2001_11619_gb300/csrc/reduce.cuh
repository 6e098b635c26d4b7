// Block-level reductions that keep FP64 work off the critical path.
//
// Pivot searches compare non-negative doubles (column norms, |entries|):
// the IEEE bit pattern of a non-negative double orders like its value, so
// the comparisons run on 64-bit integer keys (integer pipe) instead of FP64
// compares, which on this GPU share the narrow FP64 pipe.  NaN maps below
// every number, so it is never chosen.  After the warp-level shuffles only
// warp 0 combines the per-warp results and broadcasts them through shared
// memory (no thread repeats the cross-warp loop).
#pragma once

#include <cstdint>

namespace skel {

// key of |x| (or of x >= 0): its bits; NaN and negative values -> -1
__device__ __forceinline__ long long amax_key(double v) {
  const long long b = __double_as_longlong(v);
  return (b < 0 || b > 0x7FF0000000000000LL) ? -1LL : b;
}

__device__ __forceinline__ double amax_value(long long key) {
  return key < 0 ? -1.0 : __longlong_as_double(key);
}

// (key, idx) is better than (k2, i2): larger key, ties to the lower index
__device__ __forceinline__ bool amax_better(long long k, int i, long long k2,
                                            int i2) {
  return k > k2 || (k == k2 && i < i2);
}

__device__ __forceinline__ void warp_amax(long long &k, int &i) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (amax_better(k2, i2, k, i)) {
      k = k2;
      i = i2;
    }
  }
}

// Block-wide argmax of per-thread candidates (v >= 0, idx); a thread
// without a candidate passes v < 0 and an index past the valid range.
// Every thread receives the winner (v = -1 and the smallest such index
// when no thread had a candidate).  sk/si: shared arrays of NW + 1 entries
// (the last one carries the broadcast).
// Lead = false drops the leading barrier, for callers that pass another
// barrier between two calls (the slots of the previous call are read by
// then).
template <int NW, bool Lead = true>
__device__ __forceinline__ void block_amax(double &v, int &idx,
                                           long long *sk, int *si) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long k = amax_key(v);
  int i = idx;
  warp_amax(k, i);
  if (Lead) __syncthreads();  // the slots may still be read by a previous call
  if (lane == 0) {
    sk[warp] = k;
    si[warp] = i;
  }
  __syncthreads();
  if (warp == 0) {
    long long k2 = lane < NW ? sk[lane] : -1LL;
    int i2 = lane < NW ? si[lane] : 0x7fffffff;
    warp_amax(k2, i2);
    if (lane == 0) {
      sk[NW] = k2;
      si[NW] = i2;
    }
  }
  __syncthreads();
  v = amax_value(sk[NW]);
  idx = si[NW];
}

// Block-wide FP64 sum; every thread receives it.  s: NW + 1 shared doubles.
template <int NW>
__device__ __forceinline__ double block_sum_w0(double v, double *s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) s[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NW ? s[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s[NW] = t;
  }
  __syncthreads();
  return s[NW];
}

// Block-wide sum of per-thread partial sums held in Real: each warp adds
// its lanes in Real, warp 0 adds the NW warp totals in FP64.  With Real =
// float that is one FP64 step per warp instead of a full FP64 butterfly in
// every warp.  s: NW + 1 shared doubles; every thread receives the sum.
template <int NW, class Real>
__device__ __forceinline__ double block_sum_rf(Real v, double *s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) s[warp] = (double)v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NW ? s[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s[NW] = t;
  }
  __syncthreads();
  return s[NW];
}

}  // namespace skel
