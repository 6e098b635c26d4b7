// Householder building blocks shared by the one-CTA and the cluster
// column-pivoted QR kernels (FP64).
#pragma once

#include "kmath.cuh"

namespace skel {

__device__ __forceinline__ double qr_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sqrt(eps): the downdated squared norm is recomputed once it keeps less
// than this fraction of the squared norm at its last recomputation (the
// cancellation safeguard of LAPACK's xLAQP2).
constexpr double kTol3z = 1.4901161193847656e-08;

// Apply H = I - tau v v^T to columns col(q), q in [0, nq) (skipping those
// with skip(q)), rows j..m-1 of the column-major A (ld m).  v is held in
// shared memory (vs[j..m)).  Each warp streams U columns at once.
// Norm bookkeeping: on entry cn[q] is the squared norm of rows j..m-1 of
// column q, which the reflection leaves unchanged; on exit it is the squared
// norm of rows j+1..m-1, i.e. cn[q] - R_jq^2, or a fresh sum of squares when
// that downdate has cancelled below kTol3z of cn0[q] (the squared norm at
// the last recomputation, updated alongside).
template <int U, class ColFn, class SkipFn>
__device__ void apply_reflector(double *A, int m, int j, const double *vs,
                                double tau, int nq, ColFn col, SkipFn skip,
                                double *cn, double *cn0, int warp, int nwarp,
                                int lane) {
  const double vj = vs[j];
  for (int q0 = warp * U; q0 < nq; q0 += nwarp * U) {
    double *a[U];
    bool ok[U];
    double dot[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u;
      ok[u] = q < nq && !skip(q);
      a[u] = A + (int64_t)(ok[u] ? col(q) : 0) * m;
      dot[u] = 0.0;
    }
    for (int i = j + lane; i < m; i += 32) {
      const double vi = vs[i];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) dot[u] += vi * __ldcg(a[u] + i);
    }
    double sc[U], keep[U];
    bool rec[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      dot[u] = qr_warp_sum(dot[u]);
      sc[u] = tau * dot[u];
      rec[u] = false;
      keep[u] = 0.0;
      if (ok[u]) {
        const double rjc = __ldcg(a[u] + j) - sc[u] * vj;
        const double c2 = cn[q0 + u];
        double t = c2 > 0.0 ? 1.0 - rjc * rjc / c2 : 0.0;
        t = t > 0.0 ? t : 0.0;
        const double c0 = cn0[q0 + u];
        rec[u] = !(c0 > 0.0) || t * (c2 / c0) <= kTol3z;
        keep[u] = c2 * t;
      }
    }
    double nn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) nn[u] = 0.0;
    for (int i = j + lane; i < m; i += 32) {
      const double vi = vs[i];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) {
          const double x = __ldcg(a[u] + i) - sc[u] * vi;
          a[u][i] = x;
          if (rec[u] && i > j) nn[u] += x * x;
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      if (rec[u]) {
        nn[u] = qr_warp_sum(nn[u]);
        if (lane == 0) {
          cn[q0 + u] = nn[u];
          cn0[q0 + u] = nn[u];
        }
      } else if (lane == 0) {
        cn[q0 + u] = keep[u];
      }
    }
  }
}

}  // namespace skel
