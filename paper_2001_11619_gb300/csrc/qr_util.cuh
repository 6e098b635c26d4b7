// Householder building blocks shared by the one-CTA and the cluster
// column-pivoted QR kernels.  The matrix is stored in Real (double for the
// FP64 form, float for the mixed form).  The column norms, their downdates,
// the pivot choice, the stopping test and the reflector scalars are FP64;
// the dot products of a reflector with the columns and the partial sums of
// squares within a warp are in Real.  In the mixed form FP64 is ~60x
// dearer than FP32 and is charged per warp instruction, so every FP64 step
// is arranged to serve many columns or many partial sums at once.
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

// warp sum in the storage type (the dot products of the reflector: their
// per-lane partial sums are already in that type)
template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


// Apply H = I - tau v v^T to columns col(q), q in [0, nq) (skipping those
// with skip(q)), rows j..m-1 of the column-major A (ld m).  v is held in
// shared memory (vs[j..m)).  Called by every thread of the CTA (it has
// barriers); each warp streams U columns at once.
// Norm bookkeeping: on entry cn[q] is the squared norm of rows j..m-1 of
// column q, which the reflection leaves unchanged; on exit it is the squared
// norm of rows j+1..m-1, i.e. cn[q] - R_jq^2, or a fresh sum of squares when
// that downdate has cancelled below Tol3z<Real> of cn0[q] (the squared norm at
// the last recomputation, updated alongside).
// The FP64 pipe is the scarce one on this GPU, and it is charged per warp
// instruction, however few lanes are active.  So the reflection itself runs
// in the storage type, and the FP64 downdate runs afterwards with one
// thread per column (one FP64 instruction serves 32 columns), from the new
// row-j entries left in rj[q].  flag[q] marks the columns to recompute.
// rj, flag: shared arrays of nq entries.
// U columns per warp at a time; RB rows per lane per load batch (every
// load of a batch is issued before the first use).  The number of
// dependent L2 round trips per step is 2 m / (32 RB) per column group, so
// kernels with few columns per warp (the clusters) take a larger RB.
// CG: load through L2 only (ld.global.cg), for columns that other CTAs
// write (the clusters); a one-CTA kernel loads through L1, where the
// update pass finds the columns its dot pass has just read.
template <int U, int RB, class Real, class ColFn, class SkipFn,
          bool CG = true>
__device__ void apply_reflector(Real *A, int m, int j, const Real *vs,
                                double tau, int nq, ColFn col, SkipFn skip,
                                double *cn, double *cn0, Real *rj,
                                unsigned char *flag, int warp, int nwarp,
                                int lane) {
  const Real taur = (Real)tau;
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
    // rows in batches of RB per lane: every load of a batch is issued
    // before the first use, so the L2 latency overlaps (one dependent round
    // trip per batch instead of per row)
    for (int i0 = j + lane; i0 < m; i0 += 32 * RB) {
      Real av[U][RB], vv[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + 32 * r;
        const bool in = i < m;
        vv[r] = in ? vs[i] : Real(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          av[u][r] = (in && ok[u]) ? (CG ? __ldcg(a[u] + i) : a[u][i])
                                   : Real(0);
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int u = 0; u < U; ++u) dot[u] += vv[r] * av[u][r];
    }
    Real scr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) scr[u] = taur * warp_sum_t<Real>(dot[u]);
    for (int i0 = j + lane; i0 < m; i0 += 32 * RB) {
      Real av[U][RB], vv[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + 32 * r;
        const bool in = i < m;
        vv[r] = in ? vs[i] : Real(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          av[u][r] = (in && ok[u]) ? (CG ? __ldcg(a[u] + i) : a[u][i])
                                   : Real(0);
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + 32 * r;
        if (i >= m) continue;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            const Real x = av[u][r] - scr[u] * vv[r];
            a[u][i] = x;
            if (i == j) rj[q0 + u] = x;  // the new R_jq (lane 0)
          }
      }
    }
  }
  __syncthreads();
  // FP64 downdate, one thread per column (LAPACK xLAQP2 safeguard) in
  // division-free form: the new squared norm c2 - R_jq^2, recomputed when
  // it falls to Tol3z of the squared norm at the last recomputation
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    flag[q] = 0;
    if (skip(q)) continue;
    const double rjc = (double)rj[q];
    const double c2 = cn[q];
    double d = c2 > 0.0 ? c2 - rjc * rjc : 0.0;
    d = d > 0.0 ? d : 0.0;
    const double c0 = cn0[q];
    if (!(c0 > 0.0) || d <= Tol3z<Real>::value * c0)
      flag[q] = 1;
    else
      cn[q] = d;
  }
  __syncthreads();
  // fresh sums of squares (rows j+1..m-1) where the downdate cancelled
  for (int q = warp; q < nq; q += nwarp) {
    if (!flag[q]) continue;
    const Real *ac = A + (int64_t)col(q) * m;
    Real sp = Real(0);
    for (int i = j + 1 + lane; i < m; i += 32) {
      const Real x = CG ? __ldcg(ac + i) : ac[i];
      sp += x * x;
    }
    const double s2 = qr_warp_sum((double)sp);
    if (lane == 0) {
      cn[q] = s2;
      cn0[q] = s2;
    }
  }
}

}  // namespace skel
