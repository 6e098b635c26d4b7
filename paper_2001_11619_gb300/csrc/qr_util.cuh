// Householder building blocks shared by the one-CTA and the cluster
// column-pivoted QR kernels.  The matrix is stored in Real (double for the
// FP64 form, float for the mixed form); column norms, the pivot choice, the
// stopping test and the reflector scalars are always FP64.  The dot
// products of a reflector with the columns are summed in Real, and the
// FP64 norm bookkeeping runs on one lane per column: in the mixed form FP64
// is ~60x dearer than FP32, and redundant FP64 work in every lane cost more
// than the float column updates themselves.
#pragma once

#include "kmath.cuh"

namespace skel {

__device__ __forceinline__ double qr_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sqrt(eps) of the storage type: the downdated squared norm is recomputed
// once it keeps less than this fraction of the squared norm at its last
// recomputation (the cancellation safeguard of LAPACK's xLAQP2).  With float
// storage the columns carry float rounding that the FP64 downdate does not
// see, so the float epsilon sets the threshold; with the double threshold
// the pivot norms drift, wrong pivots are chosen and the rank-revealing
// stop comes too early.
template <class Real> struct Tol3z;
template <> struct Tol3z<double> {
  static constexpr double value = 1.4901161193847656e-08;  // 2^-26
};
template <> struct Tol3z<float> {
  static constexpr double value = 3.4526698300124393e-04;  // 2^-11.5
};

// Apply H = I - tau v v^T to columns col(q), q in [0, nq) (skipping those
// with skip(q)), rows j..m-1 of the column-major A (ld m).  v is held in
// shared memory (vs[j..m)).  Each warp streams U columns at once.
// Norm bookkeeping: on entry cn[q] is the squared norm of rows j..m-1 of
// column q, which the reflection leaves unchanged; on exit it is the squared
// norm of rows j+1..m-1, i.e. cn[q] - R_jq^2, or a fresh sum of squares when
// that downdate has cancelled below Tol3z<Real> of cn0[q] (the squared norm at
// the last recomputation, updated alongside).
// warp sum in the storage type (the dot products of the reflector: their
// per-lane partial sums are already in that type)
template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kRB = 4;  // rows per lane per load batch

template <int U, class Real, class ColFn, class SkipFn>
__device__ void apply_reflector(Real *A, int m, int j, const Real *vs,
                                double tau, int nq, ColFn col, SkipFn skip,
                                double *cn, double *cn0, int warp, int nwarp,
                                int lane) {
  const double vj = (double)vs[j];
  for (int q0 = warp * U; q0 < nq; q0 += nwarp * U) {
    Real *a[U];
    bool ok[U];
    Real dot[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u;
      ok[u] = q < nq && !skip(q);
      a[u] = A + (int64_t)(ok[u] ? col(q) : 0) * m;
      dot[u] = Real(0);
    }
    // rows in batches of kRB per lane: every load of a batch is issued
    // before the first use, so the L2 latency overlaps (one dependent round
    // trip per batch instead of per row)
    for (int i0 = j + lane; i0 < m; i0 += 32 * kRB) {
      Real av[U][kRB], vv[kRB];
#pragma unroll
      for (int r = 0; r < kRB; ++r) {
        const int i = i0 + 32 * r;
        const bool in = i < m;
        vv[r] = in ? vs[i] : Real(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          av[u][r] = (in && ok[u]) ? __ldcg(a[u] + i) : Real(0);
      }
#pragma unroll
      for (int r = 0; r < kRB; ++r)
#pragma unroll
        for (int u = 0; u < U; ++u) dot[u] += vv[r] * av[u][r];
    }
    // the reflector coefficients tau (v . a) in FP64, formed on lane 0 and
    // broadcast in the storage type (in every lane they would cost more
    // FP64 issue slots than the float column update)
    double sc[U];
    Real scr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const Real d = warp_sum_t<Real>(dot[u]);
      sc[u] = lane == 0 ? tau * (double)d : 0.0;
      scr[u] = __shfl_sync(0xffffffffu, (Real)sc[u], 0);
    }
    // FP64 norm bookkeeping on lane 0 only (the other lanes only need to
    // know which columns get a fresh sum of squares)
    unsigned recm = 0;
    double keep[U];
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        keep[u] = 0.0;
        if (!ok[u]) continue;
        const double rjc = (double)__ldcg(a[u] + j) - sc[u] * vj;
        const double c2 = cn[q0 + u];
        double t = c2 > 0.0 ? 1.0 - rjc * rjc / c2 : 0.0;
        t = t > 0.0 ? t : 0.0;
        const double c0 = cn0[q0 + u];
        if (!(c0 > 0.0) || t * (c2 / c0) <= Tol3z<Real>::value)
          recm |= 1u << u;
        keep[u] = c2 * t;
      }
    }
    recm = __shfl_sync(0xffffffffu, recm, 0);
    Real nn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) nn[u] = Real(0);
    for (int i0 = j + lane; i0 < m; i0 += 32 * kRB) {
      Real av[U][kRB], vv[kRB];
#pragma unroll
      for (int r = 0; r < kRB; ++r) {
        const int i = i0 + 32 * r;
        const bool in = i < m;
        vv[r] = in ? vs[i] : Real(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          av[u][r] = (in && ok[u]) ? __ldcg(a[u] + i) : Real(0);
      }
#pragma unroll
      for (int r = 0; r < kRB; ++r) {
        const int i = i0 + 32 * r;
        if (i >= m) continue;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            const Real x = av[u][r] - scr[u] * vv[r];
            a[u][i] = x;
            if (((recm >> u) & 1u) && i > j) nn[u] += x * x;
          }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      if ((recm >> u) & 1u) {
        const double s = qr_warp_sum((double)nn[u]);
        if (lane == 0) {
          cn[q0 + u] = s;
          cn0[q0 + u] = s;
        }
      } else if (lane == 0) {
        cn[q0 + u] = keep[u];
      }
    }
  }
}

}  // namespace skel
