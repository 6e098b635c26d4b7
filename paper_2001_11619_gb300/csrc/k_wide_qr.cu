// Column-pivoted QR (interpolative decomposition, Sec. 2.2 / 2.5) of one
// large box with the whole GPU.
//
// A box of thousands of active DOFs (the 64-hole quadrant case: n = 2548,
// m = 3878 at level 1; the 1M-node case: n = 3321, m = 10958) ran its
// Householder steps on one 16-CTA cluster, 16 of the 152 SMs.  Here each
// step is two launches over the whole GPU:
//
//   pivot   (one CTA): restore the previous step's diagonal, pick the
//           column of largest remaining norm (ties to the lowest index),
//           swap it into place, recompute its norm exactly, apply the
//           relative stopping test |R_jj| <= tol |R_11|, form the
//           reflector (v in place, tau, alpha);
//   reflect (CTAs of 4 columns, rows split over 256 threads): apply
//           I - tau v v^T to the trailing columns and downdate their norms
//           with the LAPACK safeguard (the rule of the one-CTA and cluster
//           kernels).
//
// Then T = R11^{-1} R12 by a blocked back substitution in FP64.  The same
// storage and precision rules as the other CPQR kernels: the matrix in
// Real (float in the mixed form), norms, pivots and reflector scalars in
// FP64, T solved in FP64 and stored in the factor type Fac.  The rank is
// known on the device only: the host issues the steps in chunks and reads
// a stop flag back between chunks (one chunk behind), and every kernel of
// a step after the stop returns at once.
#include <algorithm>

#include "qr_util.cuh"
#include "reduce.cuh"
#include "skel_internal.h"
#include "wide_util.cuh"

namespace skel {

using namespace wide;

namespace {
constexpr int kQT = 1024;       // threads of the one-CTA pivot step
constexpr int kQW = kQT / 32;
constexpr int kRT = 256;        // threads of a reflector CTA
constexpr int kRCols = 4;       // trailing columns per reflector CTA
}  // namespace

// State of one box's factorization, on the device.
struct QrOps {
  int n, m, kmax;
  int k, stop;        // the rank, once stop = 1
  int acol;           // column whose diagonal holds v0 (-1: none)
  double alpha, tau, r11;
  double *cn, *cn0;   // squared norms (n each)
  int32_t *perm;      // column order (n)
  double *R;          // R11 in FP64 (k x k, ld k), for the T solve
  double *W;          // R12, then T, in FP64 (k x r, ld k)
};

size_t qr_ops_bytes() { return sizeof(QrOps); }

template <class Real>
__global__ void k_qr_setup(const LvlBox *lb, int q, QrOps *op, double *dws,
                           int32_t *iws, double *R, double *tws) {
  const LvlBox &B = lb[q];
  const int n = B.n;
  if (threadIdx.x == 0) {
    op->n = n;
    op->m = B.m;
    op->kmax = B.m < n ? B.m : n;
    op->k = 0;
    op->stop = 0;
    op->acol = -1;
    op->alpha = op->tau = op->r11 = 0.0;
    op->cn = dws;
    op->cn0 = dws + n;
    op->perm = iws;
    op->R = R;
    op->W = tws + B.t_off;
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) iws[c] = c;
}

// squared column norms, one warp per column (sums in Real within a warp)
template <class Real>
__global__ void k_qr_norms(const LvlBox *lb, int q, const Real *dscr,
                           QrOps *op) {
  const LvlBox &B = lb[q];
  const int n = B.n, m = B.m;
  const Real *A = dscr + B.m_off;
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= n) return;
  Real sp = Real(0);
  for (int i = lane; i < m; i += 32) {
    const Real a = A[i + (int64_t)c * m];
    sp += a * a;
  }
  const double s = (double)warp_sum_t<Real>(sp);
  if (lane == 0) {
    op->cn[c] = s;
    op->cn0[c] = s;
  }
}

template <class Real>
__global__ void __launch_bounds__(kQT)
k_qr_pivot(const LvlBox *lb, int q, Real *dscr, QrOps *op, int j,
           double tol) {
  __shared__ long long sk[kQW + 1];
  __shared__ int si[kQW + 1];
  __shared__ double sv[kQW + 1];
  if (op->stop) return;
  const int n = op->n, m = op->m;
  Real *A = dscr + lb[q].m_off;
  const int tid = threadIdx.x;
  if (tid == 0 && op->acol >= 0) {  // the previous step's R_jj
    const int c = op->acol;
    A[c + (int64_t)c * m] = (Real)op->alpha;
    op->acol = -1;
  }
  if (j >= op->kmax) {
    if (tid == 0) {
      op->k = op->kmax;
      op->stop = 1;
    }
    return;
  }
  double bv = -1.0;
  int bi = n;
  for (int c = j + tid; c < n; c += kQT) {
    const double v = op->cn[c];
    if (v > bv) {
      bv = v;
      bi = c;
    }
  }
  block_amax<kQW>(bv, bi, sk, si);
  const int p = bi;
  if (p >= n) {  // no finite norm left (NaN input)
    if (tid == 0) {
      op->k = j;
      op->stop = 1;
    }
    return;
  }
  if (p != j) {
    for (int i = tid; i < m; i += kQT) {
      const Real t = A[i + (int64_t)j * m];
      A[i + (int64_t)j * m] = A[i + (int64_t)p * m];
      A[i + (int64_t)p * m] = t;
    }
    if (tid == 0) {
      const int t = op->perm[j];
      op->perm[j] = op->perm[p];
      op->perm[p] = t;
      double tc = op->cn[j];
      op->cn[j] = op->cn[p];
      op->cn[p] = tc;
      tc = op->cn0[j];
      op->cn0[j] = op->cn0[p];
      op->cn0[p] = tc;
    }
  }
  __syncthreads();
  // exact norm of the pivot's rows j..m-1
  Real sp = Real(0);
  for (int i = j + tid; i < m; i += kQT) {
    const Real a = A[i + (int64_t)j * m];
    sp += a * a;
  }
  const double nx2 = block_sum_rf<kQW, Real>(sp, sv);
  const double nrm = sqrt(nx2);
  const double r11 = j == 0 ? nrm : op->r11;
  if (nrm == 0.0 || nrm <= tol * r11) {
    if (tid == 0) {
      op->k = j;
      op->stop = 1;
    }
    return;
  }
  if (tid == 0) {
    const double x0 = (double)A[j + (int64_t)j * m];
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    op->tau = 2.0 / (nx2 - x0 * x0 + v0 * v0);
    op->alpha = alpha;
    op->acol = j;
    if (j == 0) op->r11 = nrm;
    A[j + (int64_t)j * m] = (Real)v0;
  }
}

// One CTA per kRCols trailing columns, the rows of each column split over
// all kRT threads (so the dependent L2 round trips per step are m / kRT
// per thread, not m / 32 per warp): the dot products with v in Real per
// thread, summed across the CTA in FP64 (fixed order), the update, then
// the norm downdate of the columns in FP64 with the LAPACK safeguard and,
// where it cancelled, a fresh sum of squares of rows j+1..m-1.
template <class Real>
__global__ void __launch_bounds__(kRT)
k_qr_reflect(const LvlBox *lb, int q, Real *dscr, const QrOps *op, int j) {
  __shared__ double red[kRT / 32][kRCols];
  __shared__ double scr[kRCols];
  __shared__ Real rj[kRCols];
  __shared__ int flag[kRCols];
  if (op->stop || op->acol != j) return;
  const int n = op->n, m = op->m;
  const int q0 = j + 1 + blockIdx.x * kRCols;
  if (q0 >= n) return;
  const int nq = n - q0 < kRCols ? n - q0 : kRCols;
  Real *A = dscr + lb[q].m_off;
  const Real *v = A + (int64_t)j * m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Real *col[kRCols];
#pragma unroll
  for (int u = 0; u < kRCols; ++u)
    col[u] = A + (int64_t)(q0 + (u < nq ? u : 0)) * m;
  Real dot[kRCols];
#pragma unroll
  for (int u = 0; u < kRCols; ++u) dot[u] = Real(0);
  for (int i = j + tid; i < m; i += kRT) {
    const Real vi = v[i];
#pragma unroll
    for (int u = 0; u < kRCols; ++u)
      if (u < nq) dot[u] += vi * col[u][i];
  }
#pragma unroll
  for (int u = 0; u < kRCols; ++u) {
    const double w = (double)warp_sum_t<Real>(dot[u]);
    if (lane == 0) red[warp][u] = w;
  }
  __syncthreads();
  if (tid < nq) {
    double w = 0.0;
    for (int k = 0; k < kRT / 32; ++k) w += red[k][tid];
    scr[tid] = op->tau * w;
  }
  __syncthreads();
  Real s[kRCols];
#pragma unroll
  for (int u = 0; u < kRCols; ++u) s[u] = (Real)scr[u < nq ? u : 0];
  for (int i = j + tid; i < m; i += kRT) {
    const Real vi = v[i];
#pragma unroll
    for (int u = 0; u < kRCols; ++u)
      if (u < nq) {
        const Real x = col[u][i] - s[u] * vi;
        col[u][i] = x;
        if (i == j) rj[u] = x;  // the new R_jq
      }
  }
  __syncthreads();
  if (tid < nq) {  // FP64 downdate (LAPACK xLAQP2 safeguard)
    const double rjc = (double)rj[tid];
    const double c2 = op->cn[q0 + tid];
    double t = c2 > 0.0 ? 1.0 - rjc * rjc / c2 : 0.0;
    t = t > 0.0 ? t : 0.0;
    const double c0 = op->cn0[q0 + tid];
    flag[tid] = (!(c0 > 0.0) || t * (c2 / c0) <= Tol3z<Real>::value) ? 1 : 0;
    if (!flag[tid]) op->cn[q0 + tid] = c2 * t;
  }
  __syncthreads();
  for (int u = 0; u < nq; ++u) {
    if (!flag[u]) continue;  // uniform across the CTA
    Real sp = Real(0);
    for (int i = j + 1 + tid; i < m; i += kRT) {
      const Real x = col[u][i];
      sp += x * x;
    }
    const double w = (double)warp_sum_t<Real>(sp);
    if (lane == 0) red[warp][0] = w;
    __syncthreads();
    if (tid == 0) {
      double s2 = 0.0;
      for (int k = 0; k < kRT / 32; ++k) s2 += red[k][0];
      op->cn[q0 + u] = s2;
      op->cn0[q0 + u] = s2;
    }
    __syncthreads();
  }
}

// After the last step: the last diagonal, the rank, the permutation; R11
// and R12 copied to FP64 (R ld k, W ld k) for the T solve.
template <class Real>
__global__ void k_qr_finish(const LvlBox *lb, int q, Real *dscr, QrOps *op,
                            DevBox *boxes, int32_t *iscr) {
  const LvlBox &B = lb[q];
  Real *A = dscr + B.m_off;
  const int n = op->n, m = op->m;
  if (blockIdx.x == 0 && threadIdx.x == 0 && op->acol >= 0) {
    const int c = op->acol;
    A[c + (int64_t)c * m] = (Real)op->alpha;
  }
  const int k = op->stop ? op->k : op->kmax;
  const int r = n - k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the diagonal just restored is read below only by the thread that
  // wrote it (block 0, thread 0) or after this kernel
  for (int64_t idx = t0; idx < (int64_t)k * k; idx += stride) {
    const int i = (int)(idx % k), c = (int)(idx / k);
    op->R[idx] = (i == c && op->acol == c) ? op->alpha
                                           : (double)A[i + (int64_t)c * m];
  }
  for (int64_t idx = t0; idx < (int64_t)k * r; idx += stride) {
    const int i = (int)(idx % k), c = (int)(idx / k);
    op->W[idx] = (double)A[i + (int64_t)(k + c) * m];
  }
  for (int64_t c = t0; c < n; c += stride) iscr[B.perm_off + c] = op->perm[c];
  if (t0 == 0) boxes[B.box].k = k;
}

// W <- R11^{-1} W, block rows j0..j0+31 (one warp per column of W, lane i
// holding row j0 + i), from the last block up
__global__ void k_qr_trsm_diag(const QrOps *op, int j0) {
  const int n = op->n, k = op->stop ? op->k : op->kmax, r = n - k;
  if (j0 >= k) return;
  const int jb = k - j0 < kWNB ? k - j0 : kWNB;
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= r) return;  // whole warps
  const MV R = colmajor(op->R, k), W = colmajor(op->W, k);
  double x = lane < jb ? W.at(j0 + lane, c) : 0.0;
  for (int jj = jb - 1; jj >= 0; --jj) {
    if (lane == jj) x /= R.at(j0 + jj, j0 + jj);
    const double xj = __shfl_sync(0xffffffffu, x, jj);
    if (lane < jj) x -= R.at(j0 + lane, j0 + jj) * xj;
  }
  if (lane < jb) W.at(j0 + lane, c) = x;
}

// rows above the solved block: W[0:j0, :] -= R11[0:j0, j0:j0+jb] W[j0:.., :]
__global__ void __launch_bounds__(256) k_qr_trsm_upd(const QrOps *op, int j0) {
  const int n = op->n, k = op->stop ? op->k : op->kmax, r = n - k;
  if (j0 >= k) return;
  const int jb = k - j0 < kWNB ? k - j0 : kWNB;
  const int r0 = blockIdx.x * kWT, c0 = blockIdx.y * kWT;
  if (r0 >= j0 || c0 >= r) return;
  const MV R = colmajor(op->R, k), W = colmajor(op->W, k);
  tile_gemm(W, W, R.sub(0, j0), W.sub(j0, 0), j0, r, jb, -1.0, r0, c0);
}

template <class Fac>
__global__ void k_qr_store_t(const LvlBox *lb, int q, const QrOps *op,
                             const DevBox *boxes, Fac *fac) {
  const int n = op->n, k = op->stop ? op->k : op->kmax, r = n - k;
  Fac *T = fac + boxes[lb[q].box].fac_off + fac_T(k, r);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < (int64_t)k * r; idx += (int64_t)gridDim.x * blockDim.x)
    T[idx] = (Fac)op->W[idx];
}

// Host side: the boxes go round-robin over the streams; the steps are
// issued in chunks of kChunk, and before a box's next chunk the host
// reads its stop flag as copied after the chunk before the last (so one
// chunk of steps is always queued).
template <class Real, class Fac>
cudaError_t launch_cpqr_wide(const LvlBox *lb, const std::vector<int> &qs,
                             const std::vector<int> &ns,
                             const std::vector<int> &ms, int32_t *iscr,
                             Real *dscr, DevBox *boxes, Fac *fac,
                             double *tws, double tol, QrOps *ops,
                             double *dws, int32_t *iws, double *R,
                             const std::vector<cudaStream_t> &streams,
                             volatile int32_t *hstop,
                             const std::vector<cudaEvent_t> &events) {
  constexpr int kChunk = 32;
  const int nb = (int)qs.size(), nst = (int)streams.size();
  if (nb == 0) return cudaSuccess;
  const int nmax = *std::max_element(ns.begin(), ns.end());
  for (int b = 0; b < nb; ++b) {
    cudaStream_t s = streams[b % nst];
    QrOps *op = ops + b;
    k_qr_setup<Real><<<1, 256, 0, s>>>(
        lb, qs[b], op, dws + (int64_t)b * 2 * nmax,
        iws + (int64_t)b * nmax, R + (int64_t)(b % nst) * nmax * nmax, tws);
    k_qr_norms<Real><<<(unsigned)((ns[b] + 7) / 8), 256, 0, s>>>(
        lb, qs[b], dscr, op);
    note_launches(2);
  }
  std::vector<int> next(nb, 0), kmax(nb), chunks(nb, 0);
  std::vector<char> done(nb, 0);
  for (int b = 0; b < nb; ++b) kmax[b] = std::min(ns[b], ms[b]);
  int left = nb;
  while (left > 0) {
    for (int b = 0; b < nb; ++b) {
      if (done[b]) continue;
      cudaStream_t s = streams[b % nst];
      QrOps *op = ops + b;
      // the flag copied after the chunk before the last one
      if (chunks[b] >= 2) {
        cudaEvent_t ev = events[2 * b + (chunks[b] & 1)];
        cudaError_t e = cudaEventSynchronize(ev);
        if (e != cudaSuccess) return e;
        if (hstop[2 * b + (chunks[b] & 1)]) done[b] = 1;
      }
      if (!done[b] && next[b] >= kmax[b]) done[b] = 1;
      if (done[b]) {
        --left;
        continue;
      }
      const int j1 = std::min(next[b] + kChunk, kmax[b] + 1);
      const unsigned rg = (unsigned)((ns[b] + kRCols - 1) / kRCols);
      for (int j = next[b]; j < j1; ++j) {
        k_qr_pivot<Real><<<1, kQT, 0, s>>>(lb, qs[b], dscr, op, j, tol);
        if (j < kmax[b])
          k_qr_reflect<Real><<<rg, kRT, 0, s>>>(lb, qs[b], dscr, op, j);
        note_launches(2);
      }
      next[b] = j1;
      const int slot = 2 * b + (chunks[b] & 1);
      cudaError_t e = cudaMemcpyAsync((void *)(hstop + slot), &op->stop,
                                      sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaEventRecord(events[slot], s);
      if (e != cudaSuccess) return e;
      ++chunks[b];
    }
  }
  for (int b = 0; b < nb; ++b) {
    cudaStream_t s = streams[b % nst];
    QrOps *op = ops + b;
    const int n = ns[b];
    const int gb = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1216);
    k_qr_finish<Real><<<gb, 256, 0, s>>>(lb, qs[b], dscr, op, boxes, iscr);
    note_launches(1);
    const int nblk = (n + kWNB - 1) / kWNB;
    const unsigned tr = (unsigned)((n + kWT - 1) / kWT);
    for (int t = nblk - 1; t >= 0; --t) {
      k_qr_trsm_diag<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(
          op, t * kWNB);
      if (t > 0)
        k_qr_trsm_upd<<<dim3(tr, tr), 256, 0, s>>>(op, t * kWNB);
      note_launches(t > 0 ? 2 : 1);
    }
    k_qr_store_t<Fac><<<gb, 256, 0, s>>>(lb, qs[b], op, boxes, fac);
    note_launches(1);
  }
  return cudaGetLastError();
}

#define SKEL_INST(R, F)                                                        \
  template cudaError_t launch_cpqr_wide<R, F>(                                 \
      const LvlBox *, const std::vector<int> &, const std::vector<int> &,      \
      const std::vector<int> &, int32_t *, R *, DevBox *, F *, double *,       \
      double, QrOps *, double *, int32_t *, double *,                          \
      const std::vector<cudaStream_t> &, volatile int32_t *,                   \
      const std::vector<cudaEvent_t> &);
SKEL_INST(double, double)
SKEL_INST(float, double)
SKEL_INST(float, float)
#undef SKEL_INST

}  // namespace skel
