// Elimination of one large box with the whole GPU (FP64 factors).
//
// The boxes near the top of a tree with clustered holes reach several
// thousand active DOFs (the 64-hole quadrant workload: n = 2548, k = 618 at
// level 1).  The one-CTA and 16-CTA cluster kernels run such a box on a
// few SMs with a barrier per pivot; here every step of Eq. (tmat), the LU
// of X_RR and Eq. (schurmat) is a batch of launches over all SMs:
//
//   Kp = K(perm, perm)                        gather (skeleton first)
//   X_RS = K_RS - T^T K_SS        -> Y        tiled GEMM
//   X_SR = K_SR - K_SS T          -> Z        tiled GEMM
//   X_RR = K_RR - T^T K_SR - X_RS T -> LU     two tiled GEMMs
//   X_RR = P L U                               blocked right-looking LU
//   (flag the box when a pivot is at most kMoveRatio of the largest: the
//    Sec. 2.2 remark's move of indices from R into S follows on the host)
//   Y = U^{-1} L^{-1} P^T X_RS                 row interchanges, blocked TRSM
//   X_SS = K_SS - X_SR Y                       tiled GEMM
//   Z = X_SR U^{-1} L^{-1} P^T                 blocked TRSM on Z^T, column
//                                              interchanges
//
// The rank k is found by the CPQR on the device, so the launches are sized
// for the worst case (r, k <= n) and every kernel reads the box's sizes
// and pointers from a descriptor written on the device (WideOps); CTAs
// outside the realised sizes return at once.  The results go to the same
// factor layout as the other elimination kernels.  All arithmetic is FP64
// with fixed summation orders (run-to-run deterministic).
#include <algorithm>

#include "reduce.cuh"
#include "skel_internal.h"
#include "wide_util.cuh"

namespace skel {

using namespace wide;


// Sizes and pointers of one wide box, written on the device once the rank
// is known.
struct WideOps {
  int n, k, r;
  int skip;          // 1: the LU flagged X_RR, the rest waits for the move
  double *Kp;        // n x n, ld n: K(perm, perm)
  double *T, *Y, *Z, *LU, *XSS;
  int32_t *piv;
  double ustat[2];   // largest and smallest |pivot| of the LU
  int32_t map[1 + 4 * kWNB];
  // X_RR saved before its LU (first pass only), for the split of a flagged
  // box: diagonal-pivoting state and the list of remaining indices
  double *Xs;
  int32_t *lst, *pos;
  int nl, stop, p;
  double a, ra, first;  // this step's pivot, its reciprocal, the first
  TcJob job;  // the current product, for the tensor-core GEMM
};

size_t wide_ops_bytes() { return sizeof(WideOps); }

__global__ void k_wide_setup(const LvlBox *lb, int q, const DevBox *boxes,
                             double *fac, int32_t *ipool, double *Kp,
                             double *Xs, int32_t *iws, WideOps *ops) {
  if (threadIdx.x != 0) return;
  const LvlBox &B = lb[q];
  const DevBox &D = boxes[B.box];
  const int n = B.n, k = D.k, r = n - k;
  double *F = fac + D.fac_off;
  ops->n = n;
  ops->k = k;
  ops->r = r;
  ops->skip = 0;
  ops->Kp = Kp;
  ops->T = F + fac_T(k, r);
  ops->Y = F + fac_Y(k, r);
  ops->Z = F + fac_Z(k, r);
  ops->LU = F + fac_LU(k, r);
  ops->XSS = F + fac_XSS(k, r);
  ops->piv = ipool + D.piv_off;
  ops->ustat[0] = 0.0;
  ops->ustat[1] = INFINITY;
  ops->Xs = Xs;
  ops->lst = iws;
  ops->pos = iws + n;
}

// X_RR (r x r) copied aside before its LU overwrites it
__global__ void k_wide_save_xrr(const WideOps *ops) {
  const int64_t rr = (int64_t)ops->r * ops->r;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rr;
       i += (int64_t)gridDim.x * blockDim.x)
    ops->Xs[i] = ops->LU[i];
}

// Kp = A(perm, perm) and the box's permuted DOF list
__global__ void k_wide_gather(const LvlBox *lb, int q, const int32_t *iscr,
                              const double *dsa, const DevBox *boxes,
                              int32_t *dofs, const WideOps *ops) {
  const LvlBox &B = lb[q];
  const int n = B.n;
  const double *A = dsa + B.a_off;
  const int32_t *pm = iscr + B.perm_off;
  const int32_t *act = iscr + B.act_off;
  double *Kp = ops->Kp;
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    Kp[idx] = A[pm[i] + (int64_t)pm[j] * n];
    if (j == 0) dofs[boxes[B.box].dof_off + i] = act[pm[i]];
  }
}

enum WideGemm { WG_XRS = 0, WG_XSR, WG_XRR1, WG_XRR2, WG_XSS };

// operands of product `which` of the box
__device__ void wide_operands(const WideOps *ops, int which, MV &C, MV &C0,
                              MV &A, MV &B, int &M, int &N, int &K) {
  const int n = ops->n, k = ops->k, r = ops->r;
  double *Kp = ops->Kp;
  const MV KSS = colmajor(Kp, n), KRS = colmajor(Kp + k, n),
           KSR = colmajor(Kp + (int64_t)k * n, n),
           KRR = colmajor(Kp + k + (int64_t)k * n, n);
  const MV T = colmajor(ops->T, k), Tt = transposed(ops->T, k);
  switch (which) {
    case WG_XRS:  // X_RS = K_RS - T^T K_SS  (r x k)
      C = colmajor(ops->Y, r), C0 = KRS, A = Tt, B = KSS, M = r, N = k, K = k;
      break;
    case WG_XSR:  // X_SR = K_SR - K_SS T  (k x r)
      C = colmajor(ops->Z, k), C0 = KSR, A = KSS, B = T, M = k, N = r, K = k;
      break;
    case WG_XRR1:  // X_RR = K_RR - T^T K_SR
      C = colmajor(ops->LU, r), C0 = KRR, A = Tt, B = KSR, M = r, N = r, K = k;
      break;
    case WG_XRR2:  // X_RR -= X_RS T
      C = colmajor(ops->LU, r), C0 = C, A = colmajor(ops->Y, r), B = T, M = r,
      N = r, K = k;
      break;
    default:  // X_SS = K_SS - X_SR Y  (X_SR held in Z)
      C = colmajor(ops->XSS, k), C0 = KSS, A = colmajor(ops->Z, k),
      B = colmajor(ops->Y, r), M = k, N = k, K = r;
      break;
  }
}

__global__ void __launch_bounds__(256)
k_wide_gemm(const WideOps *ops, int which) {
  if (ops->skip) return;
  MV C, C0, A, B;
  int M, N, K;
  wide_operands(ops, which, C, C0, A, B, M, N, K);
  const int r0 = blockIdx.x * kWT, c0 = blockIdx.y * kWT;
  if (r0 >= M || c0 >= N) return;
  tile_gemm(C, C0, A, B, M, N, K, -1.0, r0, c0);
}

// the same product as a job of the 3xTF32 tensor-core GEMM (an empty job
// when the box waits for its X_RR move)
__global__ void k_wide_tcjob(WideOps *ops, int which) {
  if (threadIdx.x != 0) return;
  MV C, C0, A, B;
  int M, N, K;
  wide_operands(ops, which, C, C0, A, B, M, N, K);
  TcJob &j = ops->job;
  j.A = {A.p, A.rs, A.cs};
  j.B = {B.p, B.rs, B.cs};
  j.C0 = {C0.p, C0.rs, C0.cs};
  j.C = C.p;
  j.c_rs = C.rs;
  j.c_cs = C.cs;
  j.M = ops->skip ? 0 : M;
  j.N = ops->skip ? 0 : N;
  j.K = K;
  j.sign = -1.0;
}

// ---------------------------------------------------------------------------
// blocked LU of X_RR (r x r, ld r) in place, LAPACK convention

// the panel LU(j0:r, j0:j0+jb) factored in shared memory by one CTA
__global__ void k_wide_panel(WideOps *ops, int j0, int nb) {
  extern __shared__ double P[];
  __shared__ long long sk[33];
  __shared__ int si[33];
  if (ops->skip) return;
  const int n = ops->r;
  if (j0 >= n) return;
  const int jb = n - j0 < nb ? n - j0 : nb;
  double *A = ops->LU;
  const int ld = n;
  int32_t *piv = ops->piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rows = n - j0;
  for (int idx = tid; idx < rows * jb; idx += nt) {
    const int i = idx % rows, c = idx / rows;
    P[idx] = A[(j0 + i) + (int64_t)(j0 + c) * ld];
  }
  __syncthreads();
  double umax = ops->ustat[0], umin = ops->ustat[1];
  for (int jj = 0; jj < jb; ++jj) {
    const double *pc = P + (int64_t)jj * rows;
    double bv = -1.0;
    int bi = rows;
    for (int i = jj + tid; i < rows; i += nt) {
      const double a = fabs(pc[i]);
      if (a > bv) {
        bv = a;
        bi = i;
      }
    }
    block_amax<32>(bv, bi, sk, si);  // launched with 1024 threads
    const int p = bi < rows ? bi : jj;  // NaN column: no interchange
    if (bi >= rows) bv = 0.0;
    umax = fmax(umax, bv);
    umin = fmin(umin, bv);
    if (tid == 0) piv[j0 + jj] = j0 + p;
    if (p != jj && tid < jb) {
      const double t = P[jj + (int64_t)tid * rows];
      P[jj + (int64_t)tid * rows] = P[p + (int64_t)tid * rows];
      P[p + (int64_t)tid * rows] = t;
    }
    __syncthreads();
    const double d = pc[jj];
    if (d != 0.0) {
      const double rd = 1.0 / d;
      for (int i = jj + 1 + tid; i < rows; i += nt) P[i + (int64_t)jj * rows] *= rd;
    }
    __syncthreads();
    const int w = rows - jj - 1, cw = jb - jj - 1;
    for (int idx = tid; idx < w * cw; idx += nt) {
      const int i = jj + 1 + idx % w, c = jj + 1 + idx / w;
      P[i + (int64_t)c * rows] -= P[i + (int64_t)jj * rows] * P[jj + (int64_t)c * rows];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < rows * jb; idx += nt) {
    const int i = idx % rows, c = idx / rows;
    A[(j0 + i) + (int64_t)(j0 + c) * ld] = P[idx];
  }
  if (tid == 0) {
    ops->ustat[0] = umax;
    ops->ustat[1] = umin;
    // the panel's interchanges as one row map: (row, source row) pairs
    int rows_t[2 * kWNB], src_t[2 * kWNB], cnt = 0;
    auto slot = [&](int row) {
      for (int q = 0; q < cnt; ++q)
        if (rows_t[q] == row) return q;
      rows_t[cnt] = row;
      src_t[cnt] = row;
      return cnt++;
    };
    for (int jj = 0; jj < jb; ++jj) {
      const int a = j0 + jj, b = piv[a];
      if (a == b) continue;
      const int qa = slot(a), qb = slot(b);
      const int t = src_t[qa];
      src_t[qa] = src_t[qb];
      src_t[qb] = t;
    }
    ops->map[0] = cnt;
    for (int q = 0; q < cnt; ++q) {
      ops->map[1 + 2 * q] = rows_t[q];
      ops->map[2 + 2 * q] = src_t[q];
    }
  }
}

// columns outside the panel, one warp per column: the panel's row map,
// then (right of the panel) U12 = L11^{-1} A12 solved by shuffles
__global__ void k_wide_swap_trsm(const WideOps *ops, int j0, int nb) {
  if (ops->skip) return;
  const int n = ops->r;
  if (j0 >= n) return;
  const int jb = n - j0 < nb ? n - j0 : nb;
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int c = w < j0 ? w : w + jb;
  if (c >= n) return;  // whole warps
  double *A = ops->LU;
  const int ld = n;
  double *col = A + (int64_t)c * ld;
  const int cnt = ops->map[0];
  double v[2];
  int rr[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    rr[h] = q < cnt ? ops->map[1 + 2 * q] : -1;
    v[h] = q < cnt ? col[ops->map[2 + 2 * q]] : 0.0;
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (rr[h] >= 0) col[rr[h]] = v[h];
  __syncwarp();
  if (c < j0 + jb) return;
  double x = lane < jb ? col[j0 + lane] : 0.0;
  for (int jj = 0; jj < jb; ++jj) {
    const double xj = __shfl_sync(0xffffffffu, x, jj);
    if (lane > jj && lane < jb) x -= A[(j0 + lane) + (int64_t)(j0 + jj) * ld] * xj;
  }
  if (lane < jb) col[j0 + lane] = x;
}

// trailing update A22 -= L21 U12
__global__ void __launch_bounds__(256)
k_wide_lu_gemm(const WideOps *ops, int j0, int nb) {
  if (ops->skip) return;
  const int n = ops->r;
  if (j0 >= n) return;
  const int jb = n - j0 < nb ? n - j0 : nb;
  const int base = j0 + jb;
  const int rest = n - base;
  const int r0 = blockIdx.x * kWT, c0 = blockIdx.y * kWT;
  if (r0 >= rest || c0 >= rest) return;
  const MV A = colmajor(ops->LU, n);
  const MV C = A.sub(base, base);
  tile_gemm(C, C, A.sub(base, j0), A.sub(j0, base), rest, rest, jb, -1.0, r0,
            c0);
}

// the Sec. 2.2 move test on the LU's pivots
__global__ void k_wide_check(WideOps *ops, int32_t *flag, int q, int *status,
                             int allow_move) {
  if (threadIdx.x != 0) return;
  const int r = ops->r;
  const double umax = ops->ustat[0], umin = ops->ustat[1];
  const bool moving = allow_move && r > 0 && !(umin > kMoveRatio * umax);
  flag[q] = moving ? 1 : 0;
  ops->skip = moving ? 1 : 0;
  if (!moving && r > 0 && !(umin > 1e-14 * umax))
    atomicMin(status, SKEL_ESINGULAR);
}

// ---------------------------------------------------------------------------
// triangular solves with the LU factors, blocked by kWNB rows

enum WideTrsm { WT_Y_L = 0, WT_Y_U, WT_Z_UT, WT_Z_LT };

// the solve's right-hand sides B (r x k) and triangular factor M (r x r)
__device__ void trsm_views(const WideOps *ops, int mode, MV &B, MV &M,
                           bool &lower, bool &unit) {
  const int k = ops->k, r = ops->r;
  if (mode == WT_Y_L || mode == WT_Y_U) {
    B = colmajor(ops->Y, r);        // Y (r x k)
    M = colmajor(ops->LU, r);
    lower = mode == WT_Y_L;
    unit = lower;
  } else {
    B = transposed(ops->Z, k);      // Z^T (r x k)
    M = transposed(ops->LU, r);     // U^T (lower) or L^T (unit upper)
    lower = mode == WT_Z_UT;
    unit = !lower;
  }
}

// row interchanges P^T applied to Y's rows (forward) or P to Z's columns
// (reverse), one thread per right-hand side
__global__ void k_wide_swaps(const WideOps *ops, int on_y) {
  if (ops->skip) return;
  const int k = ops->k, r = ops->r;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= k) return;
  const int32_t *piv = ops->piv;
  if (on_y) {
    double *y = ops->Y + (int64_t)s * r;
    for (int j = 0; j < r; ++j) {
      const int p = piv[j];
      if (p != j) {
        const double t = y[j];
        y[j] = y[p];
        y[p] = t;
      }
    }
  } else {
    double *z = ops->Z + s;
    for (int j = r - 1; j >= 0; --j) {
      const int p = piv[j];
      if (p != j) {
        const double t = z[(int64_t)j * k];
        z[(int64_t)j * k] = z[(int64_t)p * k];
        z[(int64_t)p * k] = t;
      }
    }
  }
}

// diagonal block [j0, j0 + jb) of the solve, one warp per right-hand side
// (lane i holds row j0 + i)
__global__ void k_wide_trsm_diag(const WideOps *ops, int mode, int j0) {
  if (ops->skip) return;
  const int k = ops->k, r = ops->r;
  if (j0 >= r) return;
  const int jb = r - j0 < kWNB ? r - j0 : kWNB;
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= k) return;  // whole warps
  MV B, M;
  bool lower, unit;
  trsm_views(ops, mode, B, M, lower, unit);
  double x = lane < jb ? B.at(j0 + lane, s) : 0.0;
  if (lower) {
    for (int jj = 0; jj < jb; ++jj) {
      if (!unit && lane == jj) x /= M.at(j0 + jj, j0 + jj);
      const double xj = __shfl_sync(0xffffffffu, x, jj);
      if (lane > jj && lane < jb) x -= M.at(j0 + lane, j0 + jj) * xj;
    }
  } else {
    for (int jj = jb - 1; jj >= 0; --jj) {
      if (!unit && lane == jj) x /= M.at(j0 + jj, j0 + jj);
      const double xj = __shfl_sync(0xffffffffu, x, jj);
      if (lane < jj) x -= M.at(j0 + lane, j0 + jj) * xj;
    }
  }
  if (lane < jb) B.at(j0 + lane, s) = x;
}

// the rows below (lower) or above (upper) the solved block
__global__ void __launch_bounds__(256)
k_wide_trsm_upd(const WideOps *ops, int mode, int j0) {
  if (ops->skip) return;
  const int k = ops->k, r = ops->r;
  if (j0 >= r) return;
  const int jb = r - j0 < kWNB ? r - j0 : kWNB;
  MV B, M;
  bool lower, unit;
  trsm_views(ops, mode, B, M, lower, unit);
  const int lo = lower ? j0 + jb : 0;
  const int rows = lower ? r - lo : j0;
  const int r0 = blockIdx.x * kWT, c0 = blockIdx.y * kWT;
  if (r0 >= rows || c0 >= k) return;
  const MV C = B.sub(lo, 0);
  tile_gemm(C, C, M.sub(lo, j0), B.sub(j0, 0), rows, k, jb, -1.0, r0, c0);
}

// ---------------------------------------------------------------------------

// one product on the tensor cores (3xTF32) or in FP64 tiles
static cudaError_t gemm_tc(WideOps *ops, int which, int n, int *status,
                           cudaStream_t s) {
  k_wide_tcjob<<<1, 32, 0, s>>>(ops, which);
  note_launches(1);
  return launch_tc_gemm(&ops->job, n, n, status, s);
}

static void gemm(WideOps *ops, int which, int n, cudaStream_t s) {
  const unsigned t = (unsigned)((n + kWT - 1) / kWT);
  k_wide_gemm<<<dim3(t, t), 256, 0, s>>>(ops, which);
  note_launches(1);
}

// the blocked solve of mode over r <= n rows: block order forward for the
// lower factors, backward for the upper ones (the last block may be
// partial: its start is the largest multiple of kWNB below r, found on the
// device; the host walks every possible start and the kernels skip those
// at or past r)
static void trsm(WideOps *ops, int mode, int n, cudaStream_t s) {
  const bool lower = mode == WT_Y_L || mode == WT_Z_UT;
  const int nblk = (n + kWNB - 1) / kWNB;
  const unsigned tr = (unsigned)((n + kWT - 1) / kWT);
  const unsigned warps_blocks = (unsigned)((n * 32 + 255) / 256);
  for (int b = 0; b < nblk; ++b) {
    const int j0 = (lower ? b : nblk - 1 - b) * kWNB;
    k_wide_trsm_diag<<<warps_blocks, 256, 0, s>>>(ops, mode, j0);
    k_wide_trsm_upd<<<dim3(tr, tr), 256, 0, s>>>(ops, mode, j0);
    note_launches(2);
  }
}

cudaError_t launch_eliminate_wide(const LvlBox *lb, const std::vector<int> &qs,
                                  const std::vector<int> &ns,
                                  const int32_t *iscr, const double *dsa,
                                  DevBox *boxes, double *fac, int32_t *ipool,
                                  int32_t *dofs, double *Kp, double *Xs,
                                  int32_t *iws, WideOps *ops, int *status,
                                  int allow_move, int32_t *flag, bool tc,
                                  const std::vector<cudaStream_t> &streams) {
  const int nmax = qs.empty() ? 0 : *std::max_element(ns.begin(), ns.end());
  const int nst = (int)streams.size();
  for (size_t b = 0; b < qs.size(); ++b) {
    const int q = qs[b], n = ns[b];
    WideOps *op = ops + b;
    cudaStream_t s = streams[b % nst];
    double *Kpb = Kp + (int64_t)(b % nst) * nmax * nmax;
    k_wide_setup<<<1, 32, 0, s>>>(lb, q, boxes, fac, ipool, Kpb,
                                  Xs + b * (int64_t)nmax * nmax,
                                  iws + b * 2 * (int64_t)nmax, op);
    const int64_t nn = (int64_t)n * n;
    const int gb = (int)std::min<int64_t>((nn + 255) / 256, 152 * 16);
    k_wide_gather<<<gb, 256, 0, s>>>(lb, q, iscr, dsa, boxes, dofs, op);
    note_launches(2);
    if (tc) {
      for (int w : {WG_XRS, WG_XSR, WG_XRR1, WG_XRR2}) {
        cudaError_t e = gemm_tc(op, w, n, status, s);
        if (e != cudaSuccess) return e;
      }
    } else {
      gemm(op, WG_XRS, n, s);
      gemm(op, WG_XSR, n, s);
      gemm(op, WG_XRR1, n, s);
      gemm(op, WG_XRR2, n, s);
    }
    if (allow_move) {
      k_wide_save_xrr<<<152 * 4, 256, 0, s>>>(op);
      note_launches(1);
    }
    // LU of X_RR: worst case r = n panels; those at or past r return.
    // The panel (r x nb doubles) is held in shared memory.
    int nb = kWNB;
    while (nb > 1 && (size_t)n * nb * sizeof(double) > 200 * 1024) nb /= 2;
    const size_t psm = (size_t)n * nb * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(
        k_wide_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    if (e != cudaSuccess) return e;
    const unsigned tr = (unsigned)((n + kWT - 1) / kWT);
    for (int j0 = 0; j0 < n; j0 += nb) {
      k_wide_panel<<<1, 1024, psm, s>>>(op, j0, nb);
      k_wide_swap_trsm<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(op, j0, nb);
      k_wide_lu_gemm<<<dim3(tr, tr), 256, 0, s>>>(op, j0, nb);
      note_launches(3);
    }
    k_wide_check<<<1, 32, 0, s>>>(op, flag, q, status, allow_move);
    note_launches(1);
    const unsigned tb = (unsigned)((n + 127) / 128);
    k_wide_swaps<<<tb, 128, 0, s>>>(op, 1);
    note_launches(1);
    trsm(op, WT_Y_L, n, s);
    trsm(op, WT_Y_U, n, s);
    if (tc) {
      cudaError_t e = gemm_tc(op, WG_XSS, n, status, s);
      if (e != cudaSuccess) return e;
    } else {
      gemm(op, WG_XSS, n, s);
    }
    trsm(op, WT_Z_UT, n, s);
    trsm(op, WT_Z_LT, n, s);
    k_wide_swaps<<<tb, 128, 0, s>>>(op, 0);
    note_launches(1);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// X_RR conditioning split (Sec. 2.2 remark) of a flagged wide box, on the
// copy saved before the LU: Gaussian elimination with diagonal pivoting
// (largest remaining |diagonal|, ties to the lowest index), stopped when it
// is at most kMoveRatio of the first pivot; the indices left over move
// from R into S.  One pivot search (one CTA) and one rank-1 update of the
// remaining block (all SMs) per step.

__global__ void k_split_init(WideOps *ops) {
  const int r = ops->r;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    ops->lst[i] = i;
    ops->pos[i] = i;
  }
  if (threadIdx.x == 0) {
    ops->nl = r;
    ops->stop = r == 0;
    ops->first = -1.0;
  }
}

__global__ void k_split_pivot(WideOps *ops) {
  __shared__ long long sk[33];
  __shared__ int si[33];
  if (ops->stop) return;
  const int r = ops->r, nl = ops->nl;
  const double *X = ops->Xs;
  double bv = -1.0;
  int bi = r;
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    const int i = ops->lst[t];
    const double a = fabs(X[i + (int64_t)i * r]);
    if (a > bv || (a == bv && i < bi)) {
      bv = a;
      bi = i;
    }
  }
  block_amax<32>(bv, bi, sk, si);  // launched with 1024 threads
  if (threadIdx.x != 0) return;
  if (bi >= r) {  // nothing finite left
    ops->stop = 1;
    return;
  }
  const int p = bi;
  const double a = X[p + (int64_t)p * r];
  if (ops->first < 0.0) ops->first = fabs(a);
  if (!(fabs(a) > kMoveRatio * ops->first)) {
    ops->stop = 1;
    return;
  }
  // remove p from the list (the last entry takes its place)
  const int tp = ops->pos[p], last = ops->lst[nl - 1];
  ops->lst[tp] = last;
  ops->pos[last] = tp;
  ops->nl = nl - 1;
  ops->p = p;
  ops->a = a;
  ops->ra = 1.0 / a;  // one division per step, not one per entry
}

// The remaining block's rank-1 update, X_ij -= X_ip (X_pj / a): CTA rows
// (blockIdx.x) over the remaining rows, columns j strided by gridDim.y, so
// no index division per entry; row p's entry is scaled once per column.
__global__ void k_split_update(const WideOps *ops) {
  if (ops->stop) return;
  const int r = ops->r, m = ops->nl, p = ops->p;
  const double ra = ops->ra;
  double *X = ops->Xs;
  const int32_t *lst = ops->lst;
  for (int jj = blockIdx.y; jj < m; jj += gridDim.y) {
    const int j = lst[jj];
    const double f = X[p + (int64_t)j * r] * ra;
    double *xj = X + (int64_t)j * r;
    const double *xp = X + (int64_t)p * r;
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < m;
         ii += gridDim.x * blockDim.x) {
      const int i = lst[ii];
      xj[i] -= xp[i] * f;
    }
  }
}

__global__ void k_split_finish(const WideOps *ops, int q,
                               const DevBox *boxes, const LvlBox *lb,
                               int32_t *ipool, int32_t *moves) {
  if (threadIdx.x != 0) return;
  const int r = ops->r, nl = ops->nl;
  int32_t *out = ipool + boxes[lb[q].box].piv_off;
  int c = 0;
  for (int i = 0; i < r; ++i)
    if (ops->pos[i] < nl && ops->lst[ops->pos[i]] == i) out[c++] = i;
  moves[q] = c;
}

cudaError_t launch_xrr_split_wide(const LvlBox *lb,
                                  const std::vector<int> &qs,
                                  const std::vector<int> &ns,
                                  const std::vector<int> &bidx,
                                  const DevBox *boxes, int32_t *ipool,
                                  WideOps *ops, int32_t *moves,
                                  const std::vector<cudaStream_t> &streams) {
  const size_t nb = qs.size(), nst = streams.size();
  int most = 0;
  for (size_t b = 0; b < nb; ++b) {
    k_split_init<<<1, 256, 0, streams[b % nst]>>>(ops + bidx[b]);
    note_launches(1);
    most = std::max(most, ns[b]);
  }
  // worst case r = n steps per box; the kernels return once the split
  // stopped.  The boxes' steps are enqueued in turn so that their streams
  // run side by side.
  for (int step = 0; step < most; ++step)
    for (size_t b = 0; b < nb; ++b) {
      if (step >= ns[b]) continue;
      WideOps *op = ops + bidx[b];
      cudaStream_t s = streams[b % nst];
      k_split_pivot<<<1, 1024, 0, s>>>(op);
      k_split_update<<<dim3(4, 304), 256, 0, s>>>(op);
      note_launches(2);
    }
  for (size_t b = 0; b < nb; ++b) {
    k_split_finish<<<1, 32, 0, streams[b % nst]>>>(ops + bidx[b], qs[b],
                                                   boxes, lb, ipool, moves);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace skel
