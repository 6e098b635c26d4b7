// Factored solve kernels (Eq. kinv, Sec. 2.7 last paragraph, Sec. 3.2):
//   * level sweeps applying U / V (and V^T / U^T for the adjoint) box by
//     box, every box of a level on disjoint DOFs, one CTA per box;
//   * the bordered top block of Eq. (partition) and its dense LU;
//   * masked reductions over the redundant rows for the coupling terms.
// All FP64.
#include "kmath.cuh"

namespace skel {

constexpr int kSweepThreads = 256;

// b_R <- X_RR^{-1} b_R (trans = 0) or X_RR^{-T} b_R (trans = 1) for one box,
// b addressed through the DOF list R (column q at offset ld q).
__device__ void lu_solve_rows(const double *LU, const int32_t *piv, int r,
                              const int32_t *R, double *b, int64_t ld,
                              int nrhs, int trans) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!trans) {
    for (int q = tid; q < nrhs; q += nt)
      for (int j = 0; j < r; ++j) {
        int p = piv[j];
        if (p != j) {
          double t = b[R[j] + ld * q];
          b[R[j] + ld * q] = b[R[p] + ld * q];
          b[R[p] + ld * q] = t;
        }
      }
    __syncthreads();
    for (int j = 0; j < r; ++j) {
      const int w = r - j - 1;
      for (int idx = tid; idx < w * nrhs; idx += nt) {
        int i = j + 1 + idx % w, q = idx / w;
        b[R[i] + ld * q] -= LU[i + (int64_t)j * r] * b[R[j] + ld * q];
      }
      __syncthreads();
    }
    for (int j = r - 1; j >= 0; --j) {
      const double d = LU[j + (int64_t)j * r];
      for (int q = tid; q < nrhs; q += nt) b[R[j] + ld * q] /= d;
      __syncthreads();
      for (int idx = tid; idx < j * nrhs; idx += nt) {
        int i = idx % j, q = idx / j;
        b[R[i] + ld * q] -= LU[i + (int64_t)j * r] * b[R[j] + ld * q];
      }
      __syncthreads();
    }
  } else {
    // X^T = U^T L^T P: forward with U^T, backward with L^T, swaps reversed
    for (int j = 0; j < r; ++j) {
      const double d = LU[j + (int64_t)j * r];
      for (int q = tid; q < nrhs; q += nt) b[R[j] + ld * q] /= d;
      __syncthreads();
      const int w = r - j - 1;
      for (int idx = tid; idx < w * nrhs; idx += nt) {
        int i = j + 1 + idx % w, q = idx / w;
        b[R[i] + ld * q] -= LU[j + (int64_t)i * r] * b[R[j] + ld * q];
      }
      __syncthreads();
    }
    for (int j = r - 1; j >= 0; --j) {
      for (int idx = tid; idx < j * nrhs; idx += nt) {
        int i = idx % j, q = idx / j;
        b[R[i] + ld * q] -= LU[j + (int64_t)i * r] * b[R[j] + ld * q];
      }
      __syncthreads();
    }
    for (int q = tid; q < nrhs; q += nt)
      for (int j = r - 1; j >= 0; --j) {
        int p = piv[j];
        if (p != j) {
          double t = b[R[j] + ld * q];
          b[R[j] + ld * q] = b[R[p] + ld * q];
          b[R[p] + ld * q] = t;
        }
      }
    __syncthreads();
  }
}

__global__ void k_up_sweep(const DevBox *boxes, const int32_t *ids,
                           const int32_t *dofs, const double *fac,
                           const int32_t *ipool, double *b, int64_t ld,
                           int nrhs, double *pre, int mode) {
  const DevBox D = boxes[ids[blockIdx.x]];
  const int n = D.n, k = D.k, r = n - k;
  if (r == 0) return;
  const int32_t *S = dofs + D.dof_off, *R = S + k;
  const double *F = fac + D.fac_off;
  const double *T = F + fac_T(k, r), *Y = F + fac_Y(k, r), *Z = F + fac_Z(k, r);
  const int tid = threadIdx.x;
  // L_T (or R_T^T): b_R -= T^T b_S
  for (int idx = tid; idx < r * nrhs; idx += kSweepThreads) {
    int i = idx % r, q = idx / r;
    double acc = 0.0;
    for (int t = 0; t < k; ++t) acc += T[t + (int64_t)i * k] * b[S[t] + ld * q];
    b[R[i] + ld * q] -= acc;
  }
  __syncthreads();
  // G_L (b_S -= Z b_R) or G_R^T (b_S -= Y^T b_R)
  for (int idx = tid; idx < k * nrhs; idx += kSweepThreads) {
    int s = idx % k, q = idx / k;
    double acc = 0.0;
    if (mode == 0)
      for (int i = 0; i < r; ++i) acc += Z[s + (int64_t)i * k] * b[R[i] + ld * q];
    else
      for (int i = 0; i < r; ++i) acc += Y[i + (int64_t)s * r] * b[R[i] + ld * q];
    b[S[s] + ld * q] -= acc;
  }
  __syncthreads();
  if (pre)
    for (int idx = tid; idx < r * nrhs; idx += kSweepThreads) {
      int i = idx % r, q = idx / r;
      pre[R[i] + ld * q] = b[R[i] + ld * q];
    }
  lu_solve_rows(F + fac_LU(k, r), ipool + D.piv_off, r, R, b, ld, nrhs, mode);
}

void launch_up_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                     const int32_t *dofs, const double *fac,
                     const int32_t *ipool, double *b, int64_t ld, int nrhs,
                     double *pre, int mode, int, cudaStream_t s) {
  if (nbox == 0 || nrhs == 0) return;
  k_up_sweep<<<nbox, kSweepThreads, 0, s>>>(boxes, ids, dofs, fac, ipool, b, ld,
                                            nrhs, pre, mode);
  note_launches(1);
}

__global__ void k_down_sweep(const DevBox *boxes, const int32_t *ids,
                             const int32_t *dofs, const double *fac, double *x,
                             int64_t ld, int nrhs, int mode) {
  const DevBox D = boxes[ids[blockIdx.x]];
  const int n = D.n, k = D.k, r = n - k;
  if (r == 0) return;
  const int32_t *S = dofs + D.dof_off, *R = S + k;
  const double *F = fac + D.fac_off;
  const double *T = F + fac_T(k, r), *Y = F + fac_Y(k, r), *Z = F + fac_Z(k, r);
  const int tid = threadIdx.x;
  // G_R (x_R -= Y x_S) or G_L^T (x_R -= Z^T x_S)
  for (int idx = tid; idx < r * nrhs; idx += kSweepThreads) {
    int i = idx % r, q = idx / r;
    double acc = 0.0;
    if (mode == 0)
      for (int t = 0; t < k; ++t) acc += Y[i + (int64_t)t * r] * x[S[t] + ld * q];
    else
      for (int t = 0; t < k; ++t) acc += Z[t + (int64_t)i * k] * x[S[t] + ld * q];
    x[R[i] + ld * q] -= acc;
  }
  __syncthreads();
  // R_T (or L_T^T): x_S -= T x_R
  for (int idx = tid; idx < k * nrhs; idx += kSweepThreads) {
    int s = idx % k, q = idx / k;
    double acc = 0.0;
    for (int i = 0; i < r; ++i) acc += T[s + (int64_t)i * k] * x[R[i] + ld * q];
    x[S[s] + ld * q] -= acc;
  }
}

void launch_down_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                       const int32_t *dofs, const double *fac, double *x,
                       int64_t ld, int nrhs, int mode, int, cudaStream_t s) {
  if (nbox == 0 || nrhs == 0) return;
  k_down_sweep<<<nbox, kSweepThreads, 0, s>>>(boxes, ids, dofs, fac, x, ld,
                                              nrhs, mode);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// out = A_R^T B_R over the rows with rmask set (A, B: rows x cols, ld),
// two-stage deterministic reduction through `partial`.
constexpr int kGramRows = 1024;

__global__ void k_gram_partial(const double *A, const double *B, int64_t rows,
                               int64_t ld, int cols, const uint8_t *rmask,
                               double *partial) {
  int64_t r0 = (int64_t)blockIdx.x * kGramRows;
  int64_t r1 = r0 + kGramRows < rows ? r0 + kGramRows : rows;
  double *out = partial + (int64_t)blockIdx.x * cols * cols;
  for (int idx = threadIdx.x; idx < cols * cols; idx += blockDim.x) {
    int a = idx % cols, c = idx / cols;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r)
      if (rmask[r]) acc += A[r + ld * a] * B[r + ld * c];
    out[idx] = acc;
  }
}

__global__ void k_sum_partials(const double *partial, int nchunk, int len,
                               double *out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len) return;
  double acc = 0.0;
  for (int c = 0; c < nchunk; ++c) acc += partial[(int64_t)c * len + idx];
  out[idx] = acc;
}

void launch_gram_masked(const double *A, const double *B, int64_t rows,
                        int64_t ld, int cols, const uint8_t *rmask,
                        double *partial, double *out, cudaStream_t s) {
  if (cols == 0) return;
  int nchunk = (int)((rows + kGramRows - 1) / kGramRows);
  k_gram_partial<<<nchunk, 256, 0, s>>>(A, B, rows, ld, cols, rmask, partial);
  note_launches(1);
  int len = cols * cols;
  k_sum_partials<<<(len + 255) / 256, 256, 0, s>>>(partial, nchunk, len, out);
  note_launches(1);
}

// top = [[A_root (already written), UH_S], [QT_S^T, -I - G]]
__global__ void k_top_fill(double *top, int ld, int s, int p3,
                           const int32_t *root_act, const double *UH,
                           const double *QT, int64_t ldh, const double *G) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)s * p3;
  if (idx < tot) {
    int i = (int)(idx % s), c = (int)(idx / s);
    top[i + (int64_t)(s + c) * ld] = UH[root_act[i] + ldh * c];
    top[(s + c) + (int64_t)i * ld] = QT[root_act[i] + ldh * c];
  }
  if (idx < (int64_t)p3 * p3) {
    int a = (int)(idx % p3), b = (int)(idx / p3);
    top[(s + a) + (int64_t)(s + b) * ld] = -(a == b ? 1.0 : 0.0) - G[a + p3 * b];
  }
}

void launch_top_fill(double *top, int ld, int s, int p3, const int32_t *root_act,
                     const double *UH, const double *QT, int64_t ldh,
                     const double *G, cudaStream_t st) {
  int64_t tot = (int64_t)s * p3;
  if ((int64_t)p3 * p3 > tot) tot = (int64_t)p3 * p3;
  if (tot == 0) return;
  k_top_fill<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(top, ld, s, p3,
                                                            root_act, UH, QT,
                                                            ldh, G);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// dense LU with partial pivoting (LAPACK convention), one column at a time:
// a 1-CTA pivot/scale kernel, then a grid-wide swap + rank-1 update.
__global__ void k_lu_pivot(double *A, int n, int ld, int j, int32_t *piv,
                           double *ustat) {
  __shared__ double sv[32];
  __shared__ int si[32];
  double bv = -1.0;
  int bi = n;
  for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
    double a = fabs(A[i + (int64_t)j * ld]);
    if (a > bv) {
      bv = a;
      bi = i;
    }
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    sv[warp] = bv;
    si[warp] = bi;
  }
  __syncthreads();
  int nw = blockDim.x / 32;
  bv = sv[0];
  bi = si[0];
  for (int w = 1; w < nw; ++w)
    if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) {
      bv = sv[w];
      bi = si[w];
    }
  const int p = bi < n ? bi : j;  // NaN column: no interchange
  if (bi >= n) bv = 0.0;
  if (threadIdx.x == 0) {
    piv[j] = p;
    ustat[0] = j == 0 ? bv : fmax(ustat[0], bv);
    ustat[1] = j == 0 ? bv : fmin(ustat[1], bv);
    double t = A[j + (int64_t)j * ld];
    A[j + (int64_t)j * ld] = A[p + (int64_t)j * ld];
    A[p + (int64_t)j * ld] = t;
  }
  __syncthreads();
  const double d = A[j + (int64_t)j * ld];
  if (d != 0.0)
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      A[i + (int64_t)j * ld] /= d;
}

__global__ void k_lu_update(double *A, int n, int ld, int j,
                            const int32_t *piv) {
  const int p = piv[j];
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    if (c == j) continue;
    double *col = A + (int64_t)c * ld;
    if (threadIdx.x == 0 && p != j) {
      double t = col[j];
      col[j] = col[p];
      col[p] = t;
    }
    if (c < j) continue;
    __syncthreads();
    const double u = col[j];
    const double *l = A + (int64_t)j * ld;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) col[i] -= l[i] * u;
    __syncthreads();
  }
}

int launch_dense_lu(double *A, int n, int ld, int32_t *piv, int *,
                    cudaStream_t s) {
  // ustat lives in the two doubles after the matrix (caller allocates)
  double *ustat = A + (int64_t)ld * n;
  for (int j = 0; j < n; ++j) {
    k_lu_pivot<<<1, 1024, 0, s>>>(A, n, ld, j, piv, ustat);
    note_launches(1);
    int grid = n - 0 < 608 ? n : 608;
    k_lu_update<<<grid, 128, 0, s>>>(A, n, ld, j, piv);
    note_launches(1);
  }
  return 0;
}

// Solve with the dense LU for nrhs columns, one CTA per column.
__global__ void k_lu_solve(const double *LU, int n, int ld, const int32_t *piv,
                           double *B, int ldb, int trans) {
  double *b = B + (int64_t)ldb * blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!trans) {
    if (tid == 0)
      for (int j = 0; j < n; ++j) {
        int p = piv[j];
        if (p != j) {
          double t = b[j];
          b[j] = b[p];
          b[p] = t;
        }
      }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const double bj = b[j];
      for (int i = j + 1 + tid; i < n; i += nt) b[i] -= LU[i + (int64_t)j * ld] * bj;
      __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
      if (tid == 0) b[j] /= LU[j + (int64_t)j * ld];
      __syncthreads();
      const double bj = b[j];
      for (int i = tid; i < j; i += nt) b[i] -= LU[i + (int64_t)j * ld] * bj;
      __syncthreads();
    }
  } else {
    for (int j = 0; j < n; ++j) {
      if (tid == 0) b[j] /= LU[j + (int64_t)j * ld];
      __syncthreads();
      const double bj = b[j];
      for (int i = j + 1 + tid; i < n; i += nt) b[i] -= LU[j + (int64_t)i * ld] * bj;
      __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
      const double bj = b[j];
      for (int i = tid; i < j; i += nt) b[i] -= LU[j + (int64_t)i * ld] * bj;
      __syncthreads();
    }
    if (tid == 0)
      for (int j = n - 1; j >= 0; --j) {
        int p = piv[j];
        if (p != j) {
          double t = b[j];
          b[j] = b[p];
          b[p] = t;
        }
      }
  }
}

void launch_dense_lu_solve(const double *LU, int n, int ld, const int32_t *piv,
                           double *B, int ldb, int nrhs, int trans,
                           cudaStream_t s) {
  if (nrhs == 0 || n == 0) return;
  k_lu_solve<<<nrhs, 512, 0, s>>>(LU, n, ld, piv, B, ldb, trans);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// top-level right-hand side and back substitution (Eq. partition)

__global__ void k_top_rhs_partial(const double *b, int64_t ldb,
                                  const double *C, int64_t ldc, int p3,
                                  const uint8_t *rmask, int64_t n2,
                                  double *partial) {
  // partial[chunk][a + p3 q] = sum over chunk rows of C[r,a] b[r,q]
  int q = blockIdx.y;
  int64_t r0 = (int64_t)blockIdx.x * kGramRows;
  int64_t r1 = r0 + kGramRows < n2 ? r0 + kGramRows : n2;
  for (int a = threadIdx.x; a < p3; a += blockDim.x) {
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r)
      if (rmask[r]) acc += C[r + ldc * a] * b[r + ldb * q];
    partial[((int64_t)blockIdx.x * gridDim.y + q) * p3 + a] = acc;
  }
}

__global__ void k_top_rhs_final(const double *b, int64_t ldb, int nrhs,
                                const int32_t *root_act, int s, int p3,
                                int nchunk, const double *partial,
                                const double *gsrc, int64_t ldg, double *rhs,
                                int ldr) {
  int q = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s + p3;
       i += gridDim.x * blockDim.x) {
    if (i < s) {
      rhs[i + (int64_t)ldr * q] = b[root_act[i] + ldb * q];
    } else {
      int a = i - s;
      double acc = 0.0;
      for (int c = 0; c < nchunk; ++c)
        acc += partial[((int64_t)c * nrhs + q) * p3 + a];
      rhs[i + (int64_t)ldr * q] = gsrc[a + ldg * q] - acc;
    }
  }
}

void launch_top_rhs(const double *b, int64_t ldb, int nrhs,
                    const int32_t *root_act, int s, const double *C,
                    int64_t ldc, int p3, const uint8_t *rmask, int64_t n2,
                    const double *gsrc, int64_t ldg, double *partial,
                    double *rhs, int ldr, cudaStream_t st) {
  int nchunk = (int)((n2 + kGramRows - 1) / kGramRows);
  if (p3 > 0)
    k_top_rhs_partial<<<dim3(nchunk, nrhs), 64, 0, st>>>(b, ldb, C, ldc, p3,
                                                         rmask, n2, partial);
    note_launches(1);
  int tot = s + p3;
  k_top_rhs_final<<<dim3((tot + 255) / 256, nrhs), 256, 0, st>>>(
      b, ldb, nrhs, root_act, s, p3, nchunk, partial, gsrc, ldg, rhs, ldr);
  note_launches(1);
}

__global__ void k_top_back(double *y, int64_t ldy, const int32_t *root_act,
                           int s, const double *W, int64_t ldw, int p3,
                           const uint8_t *rmask, int64_t n2, const double *top,
                           int ldt) {
  int q = blockIdx.y;
  const double *lam = top + (int64_t)ldt * q + s;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n2;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (!rmask[r]) continue;
    double acc = 0.0;
    for (int a = 0; a < p3; ++a) acc += W[r + ldw * a] * lam[a];
    y[r + ldy * q] -= acc;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s;
       i += gridDim.x * blockDim.x)
    y[root_act[i] + ldy * q] = top[i + (int64_t)ldt * q];
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < p3;
       a += gridDim.x * blockDim.x)
    y[n2 + a + ldy * q] = lam[a];
}

void launch_top_back(double *y, int64_t ldy, int nrhs, const int32_t *root_act,
                     int s, const double *W, int64_t ldw, int p3,
                     const uint8_t *rmask, int64_t n2, const double *top,
                     int ldt, cudaStream_t st) {
  int blocks = (int)((n2 + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  k_top_back<<<dim3(blocks, nrhs), 256, 0, st>>>(y, ldy, root_act, s, W, ldw,
                                                 p3, rmask, n2, top, ldt);
  note_launches(1);
}

__global__ void k_copy_cols(const double *src, int64_t lds, double *dst,
                            int64_t ldd, int64_t rows) {
  int q = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i + ldd * q] = src[i + lds * q];
}

void launch_copy_cols(const double *src, int64_t lds, double *dst,
                      int64_t ldd, int64_t rows, int nrhs, cudaStream_t s) {
  if (rows == 0 || nrhs == 0) return;
  int blocks = (int)((rows + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  k_copy_cols<<<dim3(blocks, nrhs), 256, 0, s>>>(src, lds, dst, ldd, rows);
  note_launches(1);
}

}  // namespace skel
