// Level sweeps of the factored solve (Eq. kinv; Sec. 2.7, last paragraph:
// the block unitriangular factors of the boxes of one level act on disjoint
// DOFs, so a level is one launch with one CTA per box and chunk of
// right-hand sides).
//
// Per CTA, a chunk of Q right-hand sides of one box's b_S and b_R is
// gathered into shared memory, the box operators are applied there, and the
// chunk is scattered back:
//   up   mode 0 (U):   b_R -= T^T b_S;  b_S -= Z b_R;    b_R <- X_RR^{-1} b_R
//   up   mode 1 (V^T): b_R -= T^T b_S;  b_S -= Y^T b_R;  b_R <- X_RR^{-T} b_R
//   down mode 0 (V):   x_R -= Y x_S;    x_S -= T x_R
//   down mode 1 (U^T): x_R -= Z^T x_S;  x_S -= T x_R
// Operands read by columns (T^T, Y^T, Z^T products) use one warp per output
// row so their global loads are coalesced; the others use one thread per
// output row.  Factors are stored as Real (double, or float in the mixed
// form) and widened to FP64; vectors are FP64.
#include "kmath.cuh"

namespace skel {

constexpr int kSwT = 256;
constexpr int kSwW = kSwT / 32;

template <class Acc>
__device__ __forceinline__ Acc sw_sum(Acc v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out[i] (-)= sum_t M[t + i ld] * x[t]  for i < rows, t < len (M read by
// columns: one warp per output row)
template <int Q, class Real, class Acc>
__device__ void sub_colmajor_T(const Real *M, int64_t ld, int len, int rows,
                               const Acc *x, Acc *out, int nq) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < rows; i += kSwW) {
    Acc acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = Acc(0);
    const Real *mc = M + (int64_t)i * ld;
    // factor entries in batches of four per lane, loaded before use
    for (int t0 = lane; t0 < len; t0 += 128) {
      Acc v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        v[r] = t0 + 32 * r < len ? (Acc)mc[t0 + 32 * r] : Acc(0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int t = t0 + 32 * r;
        if (t >= len) break;
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] += v[r] * x[t * Q + q];
      }
    }
    if constexpr (Q == 16) {
      // reduce-scatter: each level halves the values a lane keeps (the
      // half picked by its lane bit) and adds its partner's copy of them;
      // lanes 2t, 2t+1 end with the total of column q(lane).  16 shuffles
      // instead of 16 full butterflies (80).
      const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4, u1 = lane & 2;
      Acc v8[8], v4[4], v2[2];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        v8[t] = (u4 ? acc[t + 8] : acc[t]) +
                __shfl_xor_sync(0xffffffffu, u4 ? acc[t] : acc[t + 8], 16);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        v4[t] = (u3 ? v8[t + 4] : v8[t]) +
                __shfl_xor_sync(0xffffffffu, u3 ? v8[t] : v8[t + 4], 8);
#pragma unroll
      for (int t = 0; t < 2; ++t)
        v2[t] = (u2 ? v4[t + 2] : v4[t]) +
                __shfl_xor_sync(0xffffffffu, u2 ? v4[t] : v4[t + 2], 4);
      Acc v1 = (u1 ? v2[1] : v2[0]) +
                  __shfl_xor_sync(0xffffffffu, u1 ? v2[0] : v2[1], 2);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
      const int q = (u4 ? 8 : 0) + (u3 ? 4 : 0) + (u2 ? 2 : 0) + (u1 ? 1 : 0);
      if (!(lane & 1) && q < nq) out[i * Q + q] -= v1;
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] = sw_sum(acc[q]);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (q < nq) out[i * Q + q] -= acc[q];
    }
  }
}

// out[s] -= sum_i M[s + i ld] * x[i]  (M read by rows across threads)
template <int Q, class Real, class Acc>
__device__ void sub_rowmajor(const Real *M, int64_t ld, int len, int rows,
                             const Acc *x, Acc *out, int nq) {
  for (int s = threadIdx.x; s < rows; s += kSwT) {
    Acc acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = Acc(0);
    for (int i0 = 0; i0 < len; i0 += 4) {
      Acc v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        v[r] = i0 + r < len ? (Acc)M[s + (int64_t)(i0 + r) * ld] : Acc(0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (i0 + r >= len) break;
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] += v[r] * x[(i0 + r) * Q + q];
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)  // compile-time indices keep acc in registers
      if (q < nq) out[s * Q + q] -= acc[q];
  }
}

// Triangular solve of one 32-row diagonal block for the columns of b kept
// by this warp (q = warp, warp + kSwW, ...).  The block is first staged in
// shared memory by all threads (sD, 32 x 33 padded: row i of the block at
// sD[i * 33], conflict-free across lanes); lane i then holds row i's entry
// of b and each step broadcasts the solved entry with a shuffle.
// M(i, c): block entry (row i, column c); by_rows: M is contiguous along
// c (stage with c fastest); lower: forward substitution, else backward;
// unit: unit diagonal.  Ends with a barrier.
template <int Q, class Acc, class Get>
__device__ __forceinline__ void sw_diag_block(Acc *b, Acc *sD, int j0,
                                              int jb, int nq, bool by_rows,
                                              bool lower, bool unit, Get M) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < 32 * 32; idx += kSwT) {
    const int i = by_rows ? idx >> 5 : idx & 31;
    const int c = by_rows ? idx & 31 : idx >> 5;
    if (i < jb && c < jb) sD[i * 33 + c] = (Acc)M(i, c);
  }
  __syncthreads();
  const Acc *row = sD + lane * 33;
  for (int q = warp; q < nq; q += kSwW) {
    Acc v = lane < jb ? b[(j0 + lane) * Q + q] : Acc(0);
    if (lower) {
      for (int c = 0; c < jb; ++c) {
        const Acc m = lane < jb ? row[c] : Acc(0);
        if (!unit && lane == c) v *= Acc(1) / m;
        const Acc xc = __shfl_sync(0xffffffffu, v, c);
        if (lane > c) v -= m * xc;
      }
    } else {
      for (int c = jb - 1; c >= 0; --c) {
        const Acc m = lane < jb ? row[c] : Acc(0);
        if (!unit && lane == c) v *= Acc(1) / m;
        const Acc xc = __shfl_sync(0xffffffffu, v, c);
        if (lane < c) v -= m * xc;
      }
    }
    if (lane < jb) b[(j0 + lane) * Q + q] = v;
  }
  __syncthreads();
}

// Column-by-column form for chunks of several right-hand sides: each step
// updates (rows left) x nq entries, enough to occupy the CTA, and every
// FP64 operation is a useful one (the sweeps over many right-hand sides are
// bound by the FP64 pipe, where idle lanes of a blocked diagonal solve
// would cost as much as busy ones).
template <int Q, class Real, class Acc>
__device__ void lu_solve_cols(const Real *LU, const int32_t *piv, int r,
                                Acc *b, int nq, int trans) {
  const int tid = threadIdx.x;
  if (!trans) {
    for (int q = tid; q < nq; q += kSwT)
      for (int j = 0; j < r; ++j) {
        const int p = piv[j];
        if (p != j) {
          Acc t = b[j * Q + q];
          b[j * Q + q] = b[p * Q + q];
          b[p * Q + q] = t;
        }
      }
    __syncthreads();
    for (int j = 0; j < r; ++j) {
      const Real *l = LU + (int64_t)j * r;
      for (int idx = tid; idx < (r - j - 1) * nq; idx += kSwT) {
        const int i = j + 1 + idx / nq, q = idx % nq;
        b[i * Q + q] -= (Acc)l[i] * b[j * Q + q];
      }
      __syncthreads();
    }
    for (int j = r - 1; j >= 0; --j) {
      const Real *u = LU + (int64_t)j * r;
      if (tid < nq) b[j * Q + tid] *= Acc(1) / (Acc)u[j];
      __syncthreads();
      for (int idx = tid; idx < j * nq; idx += kSwT) {
        const int i = idx / nq, q = idx % nq;
        b[i * Q + q] -= (Acc)u[i] * b[j * Q + q];
      }
      __syncthreads();
    }
  } else {
    // X^T = U^T L^T P
    for (int j = 0; j < r; ++j) {
      if (tid < nq) b[j * Q + tid] *= Acc(1) / (Acc)LU[j + (int64_t)j * r];
      __syncthreads();
      for (int idx = tid; idx < (r - j - 1) * nq; idx += kSwT) {
        const int i = j + 1 + idx / nq, q = idx % nq;
        b[i * Q + q] -= (Acc)LU[j + (int64_t)i * r] * b[j * Q + q];
      }
      __syncthreads();
    }
    for (int j = r - 1; j >= 0; --j) {
      for (int idx = tid; idx < j * nq; idx += kSwT) {
        const int i = idx / nq, q = idx % nq;
        b[i * Q + q] -= (Acc)LU[j + (int64_t)i * r] * b[j * Q + q];
      }
      __syncthreads();
    }
    for (int q = tid; q < nq; q += kSwT)
      for (int j = r - 1; j >= 0; --j) {
        const int p = piv[j];
        if (p != j) {
          Acc t = b[j * Q + q];
          b[j * Q + q] = b[p * Q + q];
          b[p * Q + q] = t;
        }
      }
    __syncthreads();
  }
}

// Blocked form for a single right-hand side (the latency-bound case: one
// step of the column form has only r - j entries to update).  Blocked by 32
// columns: the diagonal block is solved by shuffles
// (sw_diag_block), then every thread applies the solved block to one
// (row, column) pair of the rest as a 32-term dot product with all its
// loads independent.  Three barriers per block of 32 columns.
template <int Q, class Real, class Acc>
__device__ void lu_solve_blocked(const Real *LU, const int32_t *piv, int r,
                                 Acc *b, int nq, int trans) {
  const int tid = threadIdx.x;
  __shared__ Acc sD[32 * 33];
  auto E = [&](int i, int j) { return LU[i + (int64_t)j * r]; };  // X(i, j)
  const int last = ((r - 1) / 32) * 32;
  if (!trans) {
    // P b; L y = P b (unit lower); U x = y
    for (int q = tid; q < nq; q += kSwT)
      for (int j = 0; j < r; ++j) {
        const int p = piv[j];
        if (p != j) {
          Acc t = b[j * Q + q];
          b[j * Q + q] = b[p * Q + q];
          b[p * Q + q] = t;
        }
      }
    __syncthreads();
    for (int j0 = 0; j0 < r; j0 += 32) {
      const int jb = min(32, r - j0);
      sw_diag_block<Q>(b, sD, j0, jb, nq, false, true, true,
                       [&](int i, int c) { return E(j0 + i, j0 + c); });
      const int rows = r - j0 - jb;
      for (int idx = tid; idx < rows * nq; idx += kSwT) {
        const int i = j0 + jb + idx / nq, q = idx % nq;
        Acc acc = Acc(0);
#pragma unroll 8
        for (int c = 0; c < jb; ++c)
          acc += (Acc)E(i, j0 + c) * b[(j0 + c) * Q + q];
        b[i * Q + q] -= acc;
      }
      __syncthreads();
    }
    for (int j0 = last; j0 >= 0; j0 -= 32) {
      const int jb = min(32, r - j0);
      sw_diag_block<Q>(b, sD, j0, jb, nq, false, false, false,
                       [&](int i, int c) { return E(j0 + i, j0 + c); });
      for (int idx = tid; idx < j0 * nq; idx += kSwT) {
        const int i = idx / nq, q = idx % nq;
        Acc acc = Acc(0);
#pragma unroll 8
        for (int c = 0; c < jb; ++c)
          acc += (Acc)E(i, j0 + c) * b[(j0 + c) * Q + q];
        b[i * Q + q] -= acc;
      }
      __syncthreads();
    }
  } else {
    // X^T = U^T L^T P: U^T z = b (lower), L^T w = z (unit upper), x = P^T w;
    // row i of U^T / L^T is column i of the LU (contiguous per thread)
    for (int j0 = 0; j0 < r; j0 += 32) {
      const int jb = min(32, r - j0);
      sw_diag_block<Q>(b, sD, j0, jb, nq, true, true, false,
                       [&](int i, int c) { return E(j0 + c, j0 + i); });
      const int rows = r - j0 - jb;
      for (int idx = tid; idx < rows * nq; idx += kSwT) {
        const int i = j0 + jb + idx / nq, q = idx % nq;
        Acc acc = Acc(0);
#pragma unroll 8
        for (int c = 0; c < jb; ++c)
          acc += (Acc)E(j0 + c, i) * b[(j0 + c) * Q + q];
        b[i * Q + q] -= acc;
      }
      __syncthreads();
    }
    for (int j0 = last; j0 >= 0; j0 -= 32) {
      const int jb = min(32, r - j0);
      sw_diag_block<Q>(b, sD, j0, jb, nq, true, false, true,
                       [&](int i, int c) { return E(j0 + c, j0 + i); });
      for (int idx = tid; idx < j0 * nq; idx += kSwT) {
        const int i = idx / nq, q = idx % nq;
        Acc acc = Acc(0);
#pragma unroll 8
        for (int c = 0; c < jb; ++c)
          acc += (Acc)E(j0 + c, i) * b[(j0 + c) * Q + q];
        b[i * Q + q] -= acc;
      }
      __syncthreads();
    }
    for (int q = tid; q < nq; q += kSwT)
      for (int j = r - 1; j >= 0; --j) {
        const int p = piv[j];
        if (p != j) {
          Acc t = b[j * Q + q];
          b[j * Q + q] = b[p * Q + q];
          b[p * Q + q] = t;
        }
      }
    __syncthreads();
  }
}

// b <- X^{-1} b (trans 0) or X^{-T} b (trans 1) in shared memory, with the
// LAPACK-convention LU of X (r x r, column-major) and its interchanges.
template <int Q, class Real, class Acc>
__device__ __forceinline__ void lu_solve_shared(const Real *LU,
                                                const int32_t *piv, int r,
                                                Acc *b, int nq, int trans) {
  if constexpr (Q == 1)
    lu_solve_blocked<Q, Real>(LU, piv, r, b, nq, trans);
  else
    lu_solve_cols<Q, Real>(LU, piv, r, b, nq, trans);
}

// Acc: the arithmetic of the sweep (the vectors in shared memory); the
// right-hand sides and outputs in global memory are FP64 either way.
template <int Q, class Real, class Acc = double>
__global__ void __launch_bounds__(kSwT)
k_up(const DevBox *boxes, const int32_t *ids, const int32_t *dofs,
     const Real *fac, const int32_t *ipool, UpJobs jobs, int64_t ld,
     int nrhs, int cap, int *status, const int32_t *items) {
  // grid: x = box, y = chunk of Q right-hand sides, z = job (independent
  // right-hand-side sets swept over the same factors); or, with items, one
  // CTA per (box id, chunk, job) item
  const int bid = items ? items[3 * blockIdx.x] : ids[blockIdx.x];
  const int chunk = items ? items[3 * blockIdx.x + 1] : (int)blockIdx.y;
  const bool j1 = items ? items[3 * blockIdx.x + 2] != 0 : blockIdx.z != 0;
  const DevBox D = boxes[bid];
  const int n = D.n, k = D.k, r = n - k;
  if (r == 0 && !jobs.snap) return;
  if (n > cap) {  // launched with too little shared memory for this box
    if (threadIdx.x == 0) atomicMin(status, SKEL_ECAPACITY);
    return;
  }
  // selects, not indexes (no local copy of the parameter struct)
  double *b = j1 ? jobs.b[1] : jobs.b[0];
  double *pre = j1 ? jobs.pre[1] : jobs.pre[0];
  const int mode = j1 ? jobs.mode[1] : jobs.mode[0];
  const double *init = j1 ? jobs.init[1] : jobs.init[0];
  const double *src = (D.leaf && init) ? init : b;
  extern __shared__ double sh_raw[];
  Acc *sh = reinterpret_cast<Acc *>(sh_raw);
  Acc *bS = sh, *bR = sh + (int64_t)k * Q;
  const int32_t *S = dofs + D.dof_off, *R = S + k;
  const Real *F = fac + D.fac_off;
  const Real *T = F + fac_T(k, r), *Y = F + fac_Y(k, r), *Z = F + fac_Z(k, r);
  const Real *LU = F + fac_LU(k, r);
  const int32_t *piv = ipool + D.piv_off;
  const int q0 = chunk * Q;
  const int nq = nrhs - q0 < Q ? nrhs - q0 : Q;
  bool nz = false;
  for (int idx = threadIdx.x; idx < n * nq; idx += kSwT) {
    const int t = idx / nq, q = idx % nq;
    const int d = t < k ? S[t] : R[t - k];
    const double v = src[d + ld * (q0 + q)];
    sh[t * Q + q] = (Acc)v;
    nz |= v != 0.0;
  }
  // A chunk whose inputs are all zero has zero outputs (every step below
  // is linear): the products and the X_RR solve are skipped and the zeros
  // written as they are.  In the bordered sweeps these are the Psi columns
  // of the holes outside the box's subtree, most chunks of most boxes.
  const bool live = __syncthreads_or(nz);
  if (live) {
    sub_colmajor_T<Q, Real>(T, k, k, r, bS, bR, nq);    // b_R -= T^T b_S
    __syncthreads();
    if (mode == 0)
      sub_rowmajor<Q, Real>(Z, k, r, k, bR, bS, nq);    // b_S -= Z b_R
    else
      sub_colmajor_T<Q, Real>(Y, r, r, k, bR, bS, nq);  // b_S -= Y^T b_R
    __syncthreads();
  }
  if (pre) {
    for (int idx = threadIdx.x; idx < r * nq; idx += kSwT) {
      const int i = idx / nq, q = idx % nq;
      pre[R[i] + ld * (q0 + q)] = (double)bR[i * Q + q];
    }
    __syncthreads();  // b_R read in full before the solve rewrites it
  }
  if (live) lu_solve_shared<Q, Real>(LU, piv, r, bR, nq, mode);
  for (int idx = threadIdx.x; idx < n * nq; idx += kSwT) {
    const int t = idx / nq, q = idx % nq;
    const int d = t < k ? S[t] : R[t - k];
    b[d + ld * (q0 + q)] = (double)sh[t * Q + q];
  }
  if (jobs.snap) {  // this box's b_S output, kept for later updates
    double *sn = jobs.snap + D.snap_off + (j1 ? (int64_t)k * nrhs : 0);
    for (int idx = threadIdx.x; idx < k * nq; idx += kSwT) {
      const int t = idx / nq, q = idx % nq;
      sn[t + (int64_t)k * (q0 + q)] = (double)sh[t * Q + q];
    }
  }
}

// b_S rows of a box that is not swept again, from its snapshot, for a
// parent that is: one CTA per (box id, chunk, job) item
__global__ void k_snap_restore(const DevBox *boxes, const int32_t *items,
                               const int32_t *dofs, UpJobs jobs, int64_t ld,
                               int nrhs, int Q) {
  const int bid = items[3 * blockIdx.x];
  const int q0 = items[3 * blockIdx.x + 1] * Q;
  const bool j1 = items[3 * blockIdx.x + 2] != 0;
  const DevBox D = boxes[bid];
  const int k = D.k;
  const int nq = nrhs - q0 < Q ? nrhs - q0 : Q;
  double *b = j1 ? jobs.b[1] : jobs.b[0];
  const double *sn = jobs.snap + D.snap_off + (j1 ? (int64_t)k * nrhs : 0);
  const int32_t *S = dofs + D.dof_off;
  for (int idx = threadIdx.x; idx < k * nq; idx += blockDim.x) {
    const int t = idx / nq, q = idx % nq;
    b[S[t] + ld * (q0 + q)] = sn[t + (int64_t)k * (q0 + q)];
  }
}

template <int Q, class Real>
__global__ void __launch_bounds__(kSwT)
k_down(const DevBox *boxes, const int32_t *ids, const int32_t *dofs,
       const Real *fac, double *x, int64_t ld, int nrhs, int mode, int cap,
       int *status) {
  // grid: x = box, y = chunk of Q right-hand sides
  const DevBox D = boxes[ids[blockIdx.x]];
  const int n = D.n, k = D.k, r = n - k;
  if (r == 0) return;
  if (n > cap) {
    if (threadIdx.x == 0) atomicMin(status, SKEL_ECAPACITY);
    return;
  }
  extern __shared__ double sh[];
  double *xS = sh, *xR = sh + (int64_t)k * Q;
  const int32_t *S = dofs + D.dof_off, *R = S + k;
  const Real *F = fac + D.fac_off;
  const Real *T = F + fac_T(k, r), *Y = F + fac_Y(k, r), *Z = F + fac_Z(k, r);
  const int q0 = blockIdx.y * Q;
  const int nq = nrhs - q0 < Q ? nrhs - q0 : Q;
  for (int idx = threadIdx.x; idx < n * nq; idx += kSwT) {
    const int t = idx / nq, q = idx % nq;
    const int d = t < k ? S[t] : R[t - k];
    sh[t * Q + q] = x[d + ld * (q0 + q)];
  }
  __syncthreads();
  if (mode == 0)
    sub_rowmajor<Q, Real>(Y, r, k, r, xS, xR, nq);      // x_R -= Y x_S
  else
    sub_colmajor_T<Q, Real>(Z, k, k, r, xS, xR, nq);    // x_R -= Z^T x_S
  __syncthreads();
  sub_rowmajor<Q, Real>(T, k, r, k, xR, xS, nq);        // x_S -= T x_R
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * nq; idx += kSwT) {
    const int t = idx / nq, q = idx % nq;
    const int d = t < k ? S[t] : R[t - k];
    x[d + ld * (q0 + q)] = sh[t * Q + q];
  }
}

static void set_smem(const void *fn, size_t sm) {
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
}

// Right-hand sides per CTA: the smallest of 4, 8, 16 that holds all of
// them, halved while the launch would give fewer than two CTAs per SM (few
// large boxes near the top of the tree: there the per-box FP64 work, not
// the factor reads, bounds the sweep), and while the chunk would not fit
// in shared memory, and at most qmax (a tuning parameter).  Depends only on
// the level, nrhs and qmax, so a sweep over a level always takes the same
// path.
static int sweep_q(int nbox, int njobs, int nrhs, int max_n, int qmax) {
  if (nrhs == 1) return 1;
  int q = nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16;
  while (q > 4 && q > qmax) q >>= 1;
  while (q > 4 && (int64_t)nbox * njobs * ((nrhs + q - 1) / q) < 2 * 152)
    q >>= 1;
  while (q > 1 && (size_t)max_n * q * 8 > 200 * 1024) q = q == 4 ? 1 : q / 2;
  return q;
}

int sweep_chunk(int nbox, int njobs, int nrhs, int max_n, int qmax) {
  return sweep_q(nbox, njobs, nrhs, max_n, qmax);
}

template <int Q, class Real>
static void up_q(const DevBox *boxes, const int32_t *ids, int nbox,
                 const int32_t *dofs, const Real *fac, const int32_t *ipool,
                 const UpJobs &jobs, int njobs, int64_t ld, int nrhs,
                 int max_n, int *status, cudaStream_t s) {
  const size_t sm = (size_t)max_n * Q * 8 + 16;
  set_smem((const void *)k_up<Q, Real>, sm);
  dim3 grid(nbox, (nrhs + Q - 1) / Q, njobs);
  k_up<Q, Real><<<grid, kSwT, sm, s>>>(boxes, ids, dofs, fac, ipool, jobs, ld,
                                       nrhs, max_n, status, nullptr);
}

template <int Q, class Real, class Acc>
static void up_items_q(const DevBox *boxes, const int32_t *items, int nitems,
                       const int32_t *dofs, const Real *fac,
                       const int32_t *ipool, const UpJobs &jobs, int64_t ld,
                       int nrhs, int max_n, int *status, cudaStream_t s) {
  const size_t sm = (size_t)max_n * Q * 8 + 16;  // sized for FP64 either way
  set_smem((const void *)k_up<Q, Real, Acc>, sm);
  k_up<Q, Real, Acc><<<nitems, kSwT, sm, s>>>(boxes, nullptr, dofs, fac,
                                              ipool, jobs, ld, nrhs, max_n,
                                              status, items);
}

template <class Real, class Acc>
void launch_up_items(const DevBox *boxes, const int32_t *items, int nitems,
                     const int32_t *dofs, const Real *fac,
                     const int32_t *ipool, const UpJobs &jobs, int64_t ld,
                     int nrhs, int q, int max_n, int *status, cudaStream_t s) {
  if (nitems == 0 || nrhs == 0) return;
  switch (q) {
    case 16: up_items_q<16, Real, Acc>(boxes, items, nitems, dofs, fac, ipool,
                                       jobs, ld, nrhs, max_n, status, s);
      break;
    case 8: up_items_q<8, Real, Acc>(boxes, items, nitems, dofs, fac, ipool,
                                     jobs, ld, nrhs, max_n, status, s);
      break;
    case 4: up_items_q<4, Real, Acc>(boxes, items, nitems, dofs, fac, ipool,
                                     jobs, ld, nrhs, max_n, status, s);
      break;
    default: up_items_q<1, Real, Acc>(boxes, items, nitems, dofs, fac, ipool,
                                      jobs, ld, nrhs, max_n, status, s);
      break;
  }
  note_launches(1);
}

void launch_snap_restore(const DevBox *boxes, const int32_t *items, int nitems,
                         const int32_t *dofs, const UpJobs &jobs, int64_t ld,
                         int nrhs, int q, cudaStream_t s) {
  if (nitems == 0) return;
  k_snap_restore<<<nitems, 128, 0, s>>>(boxes, items, dofs, jobs, ld, nrhs, q);
  note_launches(1);
}

template <int Q, class Real>
static void down_q(const DevBox *boxes, const int32_t *ids, int nbox,
                   const int32_t *dofs, const Real *fac, double *x,
                   int64_t ld, int nrhs, int mode, int max_n, int *status,
                   cudaStream_t s) {
  const size_t sm = (size_t)max_n * Q * 8 + 16;
  set_smem((const void *)k_down<Q, Real>, sm);
  dim3 grid(nbox, (nrhs + Q - 1) / Q, 1);
  k_down<Q, Real><<<grid, kSwT, sm, s>>>(boxes, ids, dofs, fac, x, ld, nrhs,
                                         mode, max_n, status);
}

template <class Real>
void launch_up_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                     const int32_t *dofs, const Real *fac,
                     const int32_t *ipool, const UpJobs &jobs, int njobs,
                     int64_t ld, int nrhs, int max_n, int qmax, int *status,
                     cudaStream_t s) {
  if (nbox == 0 || nrhs == 0 || njobs == 0) return;
  switch (sweep_q(nbox, njobs, nrhs, max_n, qmax)) {
    case 16: up_q<16, Real>(boxes, ids, nbox, dofs, fac, ipool, jobs, njobs,
                            ld, nrhs, max_n, status, s); break;
    case 8: up_q<8, Real>(boxes, ids, nbox, dofs, fac, ipool, jobs, njobs,
                          ld, nrhs, max_n, status, s); break;
    case 4: up_q<4, Real>(boxes, ids, nbox, dofs, fac, ipool, jobs, njobs,
                          ld, nrhs, max_n, status, s); break;
    default: up_q<1, Real>(boxes, ids, nbox, dofs, fac, ipool, jobs, njobs,
                           ld, nrhs, max_n, status, s); break;
  }
  note_launches(1);
}

template <class Real>
void launch_down_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                       const int32_t *dofs, const Real *fac, double *x,
                       int64_t ld, int nrhs, int mode, int max_n, int qmax,
                       int *status, cudaStream_t s) {
  if (nbox == 0 || nrhs == 0) return;
  switch (sweep_q(nbox, 1, nrhs, max_n, qmax)) {
    case 16: down_q<16, Real>(boxes, ids, nbox, dofs, fac, x, ld, nrhs, mode,
                              max_n, status, s); break;
    case 8: down_q<8, Real>(boxes, ids, nbox, dofs, fac, x, ld, nrhs, mode,
                            max_n, status, s); break;
    case 4: down_q<4, Real>(boxes, ids, nbox, dofs, fac, x, ld, nrhs, mode,
                            max_n, status, s); break;
    default: down_q<1, Real>(boxes, ids, nbox, dofs, fac, x, ld, nrhs, mode,
                             max_n, status, s); break;
  }
  note_launches(1);
}

#define SKEL_INST(R)                                                           \
  template void launch_up_items<R, double>(                                    \
      const DevBox *, const int32_t *, int, const int32_t *, const R *,        \
      const int32_t *, const UpJobs &, int64_t, int, int, int, int *,          \
      cudaStream_t);                                                           \
  template void launch_up_sweep<R>(const DevBox *, const int32_t *, int,       \
                                   const int32_t *, const R *,                 \
                                   const int32_t *, const UpJobs &, int,       \
                                   int64_t, int, int, int, int *,              \
                                   cudaStream_t);                              \
  template void launch_down_sweep<R>(const DevBox *, const int32_t *, int,     \
                                     const int32_t *, const R *, double *,     \
                                     int64_t, int, int, int, int, int *,       \
                                     cudaStream_t);
SKEL_INST(double)
SKEL_INST(float)
#undef SKEL_INST
// the mixed form's bordered sweeps: FP64 factors, FP32 arithmetic
template void launch_up_items<double, float>(
    const DevBox *, const int32_t *, int, const int32_t *, const double *,
    const int32_t *, const UpJobs &, int64_t, int, int, int, int *,
    cudaStream_t);

}  // namespace skel
