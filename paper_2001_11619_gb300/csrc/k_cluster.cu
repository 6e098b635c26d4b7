// Large-box compression on a thread-block cluster, for the FP64 form (Real =
// double) and the mixed form (Real = float).
//
// Boxes near the top of the tree are few and large (hundreds of active
// DOFs, thousands of ID-matrix rows), so one CTA per box leaves most SMs
// idle.  These kernels spread one box over a cluster of kCS CTAs:
//   * CPQR: columns are owned cyclically (column c by CTA c mod kCS); each
//     Householder step exchanges the owners' pivot candidates through
//     distributed shared memory, broadcasts the reflector, and every CTA
//     updates its own columns.  Same arithmetic as the one-CTA kernel:
//     largest exact trailing norm (ties to the lowest index), stop at
//     |R_jj| <= tol |R_11|, T = R11^{-1} R12 (Sec. 2.2, Eq. gammaT).
//   * elimination: Eq. (tmat) products split across the cluster, the LU of
//     X_RR column by column with one cluster barrier pair per pivot, then
//     Y (columns) and Z (rows) solved independently per CTA (Eq. schurmat).
// Data lives in global memory (L2 resident); loads of values written by
// other CTAs use ld.global.cg so no stale L1 line is read.
#include <cooperative_groups.h>

#include "qr_util.cuh"
#include "reduce.cuh"

namespace cg = cooperative_groups;

namespace skel {

constexpr int kCS = 16;         // CTAs per cluster (non-portable size)
constexpr int kCSMid = 4;       // CTAs per cluster for mid-size boxes
// rows per lane per load batch in the reflector application: a CTA of the
// cluster owns few columns (about n/16), so each warp streams one group of
// two columns, and the steps are bound by that group's dependent L2 round
// trips; deep batches cut their number
// (float storage; the FP64 form is bound by the FP64 pipe instead, where
// the deep batches only add register pressure)
template <class Real> struct ClusterReflect {
  static constexpr int U = sizeof(Real) == 4 ? 2 : 4;
  static constexpr int RB = sizeof(Real) == 4 ? 16 : 4;
};
constexpr int kCT = 512;        // threads per CTA
constexpr int kCW = kCT / 32;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide argmax (reduce.cuh: integer keys, ties to the lowest index);
// sk, si hold kCW + 1 entries
__device__ __forceinline__ void cta_argmax(double &v, int &idx, long long *sk,
                                           int *si) {
  block_amax<kCW>(v, idx, sk, si);
}

// ---------------------------------------------------------------------------
template <int CS, class Real, class Fac>
__global__ void __launch_bounds__(kCT)
k_cpqr_cluster(const LvlBox *lb, const int32_t *sel, int32_t *iscr,
               Real *dscr, DevBox *boxes, Fac *fac, double *tws,
               double tol) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const LvlBox &B = lb[sel[blockIdx.x / CS]];
  const int n = B.n, m = B.m;
  Real *A = dscr + B.m_off;
  const int nloc = (n - rank + CS - 1) / CS;  // owned columns rank + CS q
  extern __shared__ double smem[];
  double *sdiag = smem;                          // n: R_jj (alpha of step j)
  double *cn = sdiag + n;                        // nloc
  double *cn0 = cn + nloc;                       // nloc
  Real *rj = (Real *)(cn0 + nloc);               // nloc: new row-j entries
  Real *vsm = rj + nloc;                         // m
  int *piv = (int *)(vsm + m);                   // n
  int *red = piv + n;                            // n
  unsigned char *done = (unsigned char *)(red + n);
  unsigned char *flag = done + n;                // nloc
  __shared__ double s_bv[2];
  __shared__ double s_rs[3];  // this step's norm, v0, tau
  __shared__ double rsum[kCW + 1];
  __shared__ int s_bi[2], s_r, s_gp;
  __shared__ long long rk[kCW + 1];
  __shared__ int ri[kCW + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int q = warp; q < nloc; q += kCW) {
    const Real *a = A + (int64_t)(rank + CS * q) * m;
    Real sp = Real(0);  // per-lane partial sums in the storage type
    for (int i = lane; i < m; i += 32) {
      const Real t = __ldcg(a + i);
      sp += t * t;
    }
    const double s = wsum((double)sp);
    if (lane == 0) {
      cn[q] = s;
      cn0[q] = s;
    }
  }
  for (int c = tid; c < n; c += kCT) done[c] = 0;
  __syncthreads();

  const int kmax = m < n ? m : n;
  int k = kmax;
  double r11 = 0.0;
  for (int j = 0; j < kmax; ++j) {
    double bv = -1.0;
    int bi = n;
    for (int q = tid; q < nloc; q += kCT) {
      int c = rank + CS * q;
      if (!done[c] && cn[q] > bv) {
        bv = cn[q];
        bi = c;
      }
    }
    cta_argmax(bv, bi, rk, ri);
    const int slot = j & 1;  // double buffer: a CTA may publish step j+1's
                             // candidate while another still reads step j's
    if (tid == 0) {
      s_bv[slot] = bv;
      s_bi[slot] = bi;
    }
    cl.sync();  // candidates published (the only cluster barrier per step)
    // warp 0 gathers the CS candidates (one remote load per lane) and
    // broadcasts the winner through local shared memory
    if (warp == 0) {
      long long gk = -1LL;
      int gi = n;
      if (lane < CS) {
        gk = amax_key(*cl.map_shared_rank(&s_bv[slot], lane));
        gi = *cl.map_shared_rank(&s_bi[slot], lane);
      }
      warp_amax(gk, gi);
      if (lane == 0) s_gp = gi;
    }
    __syncthreads();
    const int p = s_gp;
    if (p >= n) {  // no finite norm left
      k = j;
      break;
    }
    // Every CTA copies the pivot column into shared memory and forms its
    // exact FP64 norm (the candidates' norms are downdated estimates).  The
    // reduction order is fixed, so all CTAs get the same scalars and the
    // same stopping decision without exchanging them.  The column was last
    // written by its owner before the barrier above, and no CTA writes it
    // during this step (the diagonal alpha goes to sdiag).
    const Real *pc = A + (int64_t)p * m;
    Real sp = Real(0);  // per-thread partial sums in the storage type
    for (int i = j + tid; i < m; i += kCT) {
      const Real t = __ldcg(pc + i);
      vsm[i] = t;
      sp += t * t;
    }
    const double nx2 = block_sum_rf<kCW, Real>(sp, rsum);
    if (tid == 0) {
      const double nrm = sqrt(nx2);
      const double x0 = (double)vsm[j];
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      s_rs[0] = nrm;
      s_rs[1] = v0;
      s_rs[2] = nrm > 0.0 ? 2.0 / (nx2 - x0 * x0 + v0 * v0) : 0.0;
      sdiag[j] = alpha;
      vsm[j] = (Real)v0;
      // the same stopping test as below: a column that stops the CPQR
      // stays redundant
      const double r11j = j == 0 ? nrm : r11;
      if (nrm > 0.0 && nrm > tol * r11j) {
        piv[j] = p;
        done[p] = 1;
      }
    }
    __syncthreads();
    const double nrm = s_rs[0];
    if (j == 0) r11 = nrm;
    if (!(nrm > 0.0) || nrm <= tol * r11) {
      k = j;
      break;
    }
    const double tau = s_rs[2];
    // the owned columns are written by this CTA alone (pivoting marks
    // columns done instead of moving them), so they load through L1; the
    // pivot column and T read other CTAs' columns through L2 only
    auto own = [&](int q) { return rank + CS * q; };
    auto isdone = [&](int q) { return done[rank + CS * q] != 0; };
    apply_reflector<ClusterReflect<Real>::U, ClusterReflect<Real>::RB, Real,
                    decltype(own), decltype(isdone), false>(
        A, m, j, vsm, tau, nloc, own, isdone, cn, cn0, rj, flag, warp, kCW,
        lane);
    __syncthreads();
  }
  // every CTA reached the same k; the R factor is complete once all
  // updates of the last step have landed
  cl.sync();
  if (tid == 0) {
    int t = 0;
    for (int c = 0; c < n; ++c)
      if (!done[c]) red[t++] = c;
    s_r = t;
  }
  __syncthreads();
  const int r = s_r;  // == n - k
  DevBox &D = boxes[B.box];
  Fac *T = fac + D.fac_off + fac_T(k, r);
  double *W = tws + B.t_off;
  int32_t *po = iscr + B.perm_off;
  if (rank == 0) {
    for (int c = tid; c < k; c += kCT) po[c] = piv[c];
    for (int c = tid; c < r; c += kCT) po[k + c] = red[c];
    if (tid == 0) D.k = k;
  }
  // T = R11^{-1} R12 in FP64 (workspace W), one warp per redundant column,
  // then stored as Real
  for (int t = rank * kCW + warp; t < r; t += CS * kCW) {
    double *x = W + (int64_t)t * k;
    const Real *a = A + (int64_t)red[t] * m;
    for (int i = lane; i < k; i += 32) x[i] = (double)__ldcg(a + i);
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
      const Real *ri_col = A + (int64_t)piv[i] * m;
      double xi = 0.0;
      if (lane == 0) {
        xi = x[i] / sdiag[i];
        x[i] = xi;
      }
      xi = __shfl_sync(0xffffffffu, xi, 0);
      for (int l = lane; l < i; l += 32)
        x[l] -= (double)__ldcg(ri_col + l) * xi;
      __syncwarp();
    }
    Fac *tc = T + (int64_t)t * k;
    for (int i = lane; i < k; i += 32) tc[i] = (Fac)x[i];
  }
  cl.sync();  // no CTA leaves while its shared memory may still be read
}

// ---------------------------------------------------------------------------
template <int CS, class Real>
__global__ void __launch_bounds__(kCT)
k_eliminate_cluster(const LvlBox *lb, const int32_t *sel, const int32_t *iscr,
                    const Real *dscr, DevBox *boxes, Real *fac,
                    int32_t *ipool, int32_t *dofs, int *status,
                    int allow_move, int32_t *flag) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const LvlBox &B = lb[sel[blockIdx.x / CS]];
  DevBox &D = boxes[B.box];
  const int n = B.n, k = __ldcg(&D.k), r = n - k;
  const int tid = threadIdx.x;
  const int gt = rank * kCT + tid, gs = CS * kCT;
  const Real *A = dscr + B.a_off;
  const int32_t *act = iscr + B.act_off;
  const int32_t *perm_g = iscr + B.perm_off;
  extern __shared__ double smem[];
  double *colj = smem;                 // r
  int *pm = (int *)(colj + r);         // n
  __shared__ double rv[kCW];
  __shared__ long long rk[kCW + 1];
  __shared__ int ri[kCW + 1];
  for (int i = tid; i < n; i += kCT) pm[i] = __ldcg(perm_g + i);
  __syncthreads();
  if (rank == 0)
    for (int i = tid; i < n; i += kCT) dofs[D.dof_off + i] = act[pm[i]];
  Real *F = fac + D.fac_off;
  const Real *T = F + fac_T(k, r);
  Real *Y = F + fac_Y(k, r);
  Real *Z = F + fac_Z(k, r);
  Real *LU = F + fac_LU(k, r);
  Real *XSS = F + fac_XSS(k, r);
  int32_t *piv = ipool + D.piv_off;
#define KA(i, j) A[pm[i] + (int64_t)pm[j] * n]
#define TT(t, i) __ldcg(T + (t) + (int64_t)(i) * k)
  // Eq. (tmat): X_RS = K_RS - T^T K_SS -> Y; X_SR = K_SR - K_SS T -> Z
  for (int64_t idx = gt; idx < (int64_t)r * k; idx += gs) {
    int i = (int)(idx % r), s = (int)(idx / r);
    Real acc = KA(k + i, s);
    for (int t = 0; t < k; ++t) acc -= TT(t, i) * KA(t, s);
    Y[idx] = acc;
  }
  for (int64_t idx = gt; idx < (int64_t)k * r; idx += gs) {
    int s = (int)(idx % k), i = (int)(idx / k);
    Real acc = KA(s, k + i);
    for (int t = 0; t < k; ++t) acc -= KA(s, t) * TT(t, i);
    Z[idx] = acc;
  }
  cl.sync();
  // X_RR = K_RR - T^T K_SR - X_RS T -> LU
  for (int64_t idx = gt; idx < (int64_t)r * r; idx += gs) {
    int i = (int)(idx % r), j = (int)(idx / r);
    Real acc = KA(k + i, k + j);
    for (int t = 0; t < k; ++t)
      acc -= TT(t, i) * KA(t, k + j) + __ldcg(Y + i + (int64_t)t * r) * TT(t, j);
    LU[idx] = acc;
  }
#undef KA
  cl.sync();
  // LU of X_RR with partial pivoting; column c is handled by CTA c mod CS
  double umax = 0.0, umin = INFINITY;
  for (int j = 0; j < r; ++j) {
    double bv = -1.0;
    int bi = r;
    for (int i = j + tid; i < r; i += kCT) {
      const double a = (double)__ldcg(LU + i + (int64_t)j * r);
      colj[i] = a;
      if (fabs(a) > bv) {
        bv = fabs(a);
        bi = i;
      }
    }
    cta_argmax(bv, bi, rk, ri);
    int p = bi;
    if (p >= r) {
      p = j;
      bv = 0.0;
    }
    umax = fmax(umax, bv);
    umin = fmin(umin, bv);
    const double d = (p == j) ? colj[j] : colj[p];
    cl.sync();  // every CTA holds column j before it is rewritten
    if (p != j)
      for (int c = rank + CS * tid; c < r; c += CS * kCT) {
        if (c == j) continue;
        const Real t = __ldcg(LU + j + (int64_t)c * r);
        LU[j + (int64_t)c * r] = __ldcg(LU + p + (int64_t)c * r);
        LU[p + (int64_t)c * r] = t;
      }
    __syncthreads();
    const int w = r - j - 1;
    const int nown = (r - rank + CS - 1) / CS;
    for (int64_t idx = tid; idx < (int64_t)w * nown; idx += kCT) {
      int i = j + 1 + (int)(idx % w);
      int c = rank + CS * (int)(idx / w);
      if (c <= j) continue;
      const Real li = (Real)(((i == p) ? colj[j] : colj[i]) / d);
      LU[i + (int64_t)c * r] =
          __ldcg(LU + i + (int64_t)c * r) - li * __ldcg(LU + j + (int64_t)c * r);
    }
    if (j % CS == rank) {
      for (int i = j + 1 + tid; i < r; i += kCT)
        LU[i + (int64_t)j * r] = (Real)(((i == p) ? colj[j] : colj[i]) / d);
      if (tid == 0) {
        LU[j + (int64_t)j * r] = (Real)d;
        piv[j] = p;
      }
    }
    cl.sync();
  }
  // X_RR conditioning (Sec. 2.2 remark): flag and stop, as in k_eliminate
  const bool moving = allow_move && r > 0 && !(umin > kMoveRatio * umax);
  if (rank == 0 && tid == 0) flag[sel[blockIdx.x / CS]] = moving ? 1 : 0;
  if (moving) {
    cl.sync();
    return;
  }
  if (r > 0 && rank == 0 && tid == 0 && !(umin > 1e-14 * umax))
    atomicMin(status, SKEL_ESINGULAR);
  // Y = X_RR^{-1} X_RS: CTA rank solves the columns s = rank + CS q
  const int ny = (k - rank + CS - 1) / CS;
  for (int q = tid; q < ny; q += kCT) {
    const int s = rank + CS * q;
    for (int j = 0; j < r; ++j) {
      int p = __ldcg(piv + j);
      if (p != j) {
        const Real t = __ldcg(Y + j + (int64_t)s * r);
        Y[j + (int64_t)s * r] = __ldcg(Y + p + (int64_t)s * r);
        Y[p + (int64_t)s * r] = t;
      }
    }
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const int w = r - j - 1;
    for (int64_t idx = tid; idx < (int64_t)w * ny; idx += kCT) {
      int i = j + 1 + (int)(idx % w), s = rank + CS * (int)(idx / w);
      Y[i + (int64_t)s * r] = __ldcg(Y + i + (int64_t)s * r) -
                              __ldcg(LU + i + (int64_t)j * r) *
                                  __ldcg(Y + j + (int64_t)s * r);
    }
    __syncthreads();
  }
  for (int j = r - 1; j >= 0; --j) {
    const Real dd = __ldcg(LU + j + (int64_t)j * r);
    for (int q = tid; q < ny; q += kCT) {
      Real *yp = Y + j + (int64_t)(rank + CS * q) * r;
      *yp = __ldcg(yp) / dd;
    }
    __syncthreads();
    for (int64_t idx = tid; idx < (int64_t)j * ny; idx += kCT) {
      int i = (int)(idx % j), s = rank + CS * (int)(idx / j);
      Y[i + (int64_t)s * r] = __ldcg(Y + i + (int64_t)s * r) -
                              __ldcg(LU + i + (int64_t)j * r) *
                                  __ldcg(Y + j + (int64_t)s * r);
    }
    __syncthreads();
  }
  cl.sync();
  // Eq. (schurmat): X_SS = K_SS - X_SR Y (X_SR still in Z)
  for (int64_t idx = gt; idx < (int64_t)k * k; idx += gs) {
    int s = (int)(idx % k), t = (int)(idx / k);
    Real acc = A[pm[s] + (int64_t)pm[t] * n];
    for (int i = 0; i < r; ++i)
      acc -= __ldcg(Z + s + (int64_t)i * k) * __ldcg(Y + i + (int64_t)t * r);
    XSS[idx] = acc;
  }
  cl.sync();
  // Z = X_SR X_RR^{-1}: CTA rank solves the rows s = rank + CS q
  const int nz = ny;
  for (int j = 0; j < r; ++j) {
    const Real dd = __ldcg(LU + j + (int64_t)j * r);
    for (int q = tid; q < nz; q += kCT) {
      Real *zp = Z + (rank + CS * q) + (int64_t)j * k;
      *zp = __ldcg(zp) / dd;
    }
    __syncthreads();
    const int w = r - j - 1;
    for (int64_t idx = tid; idx < (int64_t)w * nz; idx += kCT) {
      int s = rank + CS * (int)(idx % nz), c = j + 1 + (int)(idx / nz);
      Z[s + (int64_t)c * k] = __ldcg(Z + s + (int64_t)c * k) -
                              __ldcg(Z + s + (int64_t)j * k) *
                                  __ldcg(LU + j + (int64_t)c * r);
    }
    __syncthreads();
  }
  for (int j = r - 1; j >= 0; --j) {
    for (int64_t idx = tid; idx < (int64_t)j * nz; idx += kCT) {
      int s = rank + CS * (int)(idx % nz), c = (int)(idx / nz);
      Z[s + (int64_t)c * k] = __ldcg(Z + s + (int64_t)c * k) -
                              __ldcg(Z + s + (int64_t)j * k) *
                                  __ldcg(LU + j + (int64_t)c * r);
    }
    __syncthreads();
  }
  for (int q = tid; q < nz; q += kCT) {
    const int s = rank + CS * q;
    for (int j = r - 1; j >= 0; --j) {
      int p = __ldcg(piv + j);
      if (p != j) {
        const Real t = __ldcg(Z + s + (int64_t)j * k);
        Z[s + (int64_t)j * k] = __ldcg(Z + s + (int64_t)p * k);
        Z[s + (int64_t)p * k] = t;
      }
    }
  }
#undef TT
  cl.sync();
}

static cudaError_t launch_cluster(const void *fn, int nsel, size_t smem,
                                  cudaStream_t s, void **args, int cs) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsel * cs, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  if (cs > 8)
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed,
                         1);
  return cudaLaunchKernelExC(&cfg, fn, args);
}

int cluster_size() { return kCS; }

template <class Real, class Fac>
cudaError_t launch_cpqr_cluster(const LvlBox *lb, const int32_t *sel, int nsel,
                                int32_t *iscr, Real *dscr, DevBox *boxes,
                                Fac *fac, double *tws, double tol, int max_n,
                                int max_m, cudaStream_t s, int cs) {
  if (nsel == 0) return cudaSuccess;
  size_t smem = (size_t)(max_n / cs + 1) * (16 + sizeof(Real) + 1) +
                (size_t)max_m * sizeof(Real) + (size_t)max_n * 17 + 64;
  void *args[] = {(void *)&lb,    (void *)&sel, (void *)&iscr, (void *)&dscr,
                  (void *)&boxes, (void *)&fac, (void *)&tws,  (void *)&tol};
  const void *fn = cs == kCSMid ? (const void *)k_cpqr_cluster<kCSMid, Real, Fac>
                                : (const void *)k_cpqr_cluster<kCS, Real, Fac>;
  // the rest of each SM as L1, which holds the CTA's owned columns
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxL1);
  cudaError_t e = launch_cluster(fn, nsel, smem, s, args,
                                 cs == kCSMid ? kCSMid : kCS);
  note_launches(1);
  return e;
}

template <class Real>
cudaError_t launch_eliminate_cluster(const LvlBox *lb, const int32_t *sel,
                                     int nsel, const int32_t *iscr,
                                     const Real *dscr, DevBox *boxes,
                                     Real *fac, int32_t *ipool, int32_t *dofs,
                                     int max_n, int *status, int allow_move,
                                     int32_t *flag, cudaStream_t s, int cs) {
  if (nsel == 0) return cudaSuccess;
  size_t smem = (size_t)max_n * 12 + 64;
  void *args[] = {(void *)&lb,    (void *)&sel,   (void *)&iscr,
                  (void *)&dscr,  (void *)&boxes, (void *)&fac,
                  (void *)&ipool, (void *)&dofs,  (void *)&status,
                  (void *)&allow_move, (void *)&flag};
  const void *fn = cs == kCSMid ? (const void *)k_eliminate_cluster<kCSMid, Real>
                                : (const void *)k_eliminate_cluster<kCS, Real>;
  cudaError_t e = launch_cluster(fn, nsel, smem, s, args,
                                 cs == kCSMid ? kCSMid : kCS);
  note_launches(1);
  return e;
}

// ---------------------------------------------------------------------------
// Indices to move from R into S for a box whose X_RR LU was flagged (Sec.
// 2.2 remark).  X_RR is formed again (X_RS is still in Y), then eliminated
// with diagonal pivoting: the largest remaining |diagonal| (ties to the
// lowest index) is the pivot, until it is at most kMoveRatio of the first
// pivot.  The indices left over are written ascending to the box's pivot
// slot of ipool and their number to moves[q].  Rows and columns are never
// swapped: every CTA keeps the same list of remaining indices (removal by
// swap with the last entry), and CTA c updates the columns at list
// positions c, c + kCS, ...  One cluster barrier per step.
template <int CS, class Real>
__global__ void __launch_bounds__(kCT)
k_xrr_split_cluster(const LvlBox *lb, const int32_t *sel, const int32_t *iscr,
                    const Real *dscr, DevBox *boxes, Real *fac,
                    int32_t *ipool, int32_t *moves) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int q = sel[blockIdx.x / CS];
  const LvlBox &B = lb[q];
  DevBox &D = boxes[B.box];
  const int n = B.n, k = __ldcg(&D.k), r = n - k;
  const int tid = threadIdx.x;
  const int gt = rank * kCT + tid, gs = CS * kCT;
  const Real *A = dscr + B.a_off;
  const int32_t *perm_g = iscr + B.perm_off;
  extern __shared__ double smem[];
  double *colp = smem;                 // r: column of the pivot
  int *pm = (int *)(colp + r);         // n: permutation
  int *lst = pm + n;                   // r: remaining indices
  int *pos = lst + r;                  // r: position of each index in lst
  __shared__ double rv[kCW];
  __shared__ long long rk[kCW + 1];
  __shared__ int ri[kCW + 1];
  __shared__ int s_nl;
  for (int i = tid; i < n; i += kCT) pm[i] = __ldcg(perm_g + i);
  for (int i = tid; i < r; i += kCT) {
    lst[i] = i;
    pos[i] = i;
  }
  if (tid == 0) s_nl = r;
  __syncthreads();
  Real *F = fac + D.fac_off;
  const Real *T = F + fac_T(k, r);
  const Real *Y = F + fac_Y(k, r);
  Real *X = F + fac_LU(k, r);
#define KA(i, j) A[pm[i] + (int64_t)pm[j] * n]
#define TT(t, i) __ldcg(T + (t) + (int64_t)(i) * k)
  for (int64_t idx = gt; idx < (int64_t)r * r; idx += gs) {
    int i = (int)(idx % r), j = (int)(idx / r);
    Real acc = KA(k + i, k + j);
    for (int t = 0; t < k; ++t)
      acc -= TT(t, i) * KA(t, k + j) + __ldcg(Y + i + (int64_t)t * r) * TT(t, j);
    X[idx] = acc;
  }
#undef KA
#undef TT
  cl.sync();
  double first = -1.0;
  for (int s = 0; s < r; ++s) {
    const int nl = s_nl;
    double bv = -1.0;
    int bi = r;
    for (int t = tid; t < nl; t += kCT) {
      const int i = lst[t];
      const double a = fabs((double)__ldcg(X + i + (int64_t)i * r));
      if (a > bv || (a == bv && i < bi)) {
        bv = a;
        bi = i;
      }
    }
    cta_argmax(bv, bi, rk, ri);
    if (bi >= r) break;                       // nothing finite left
    const int p = bi;
    const double a = (double)__ldcg(X + p + (int64_t)p * r);
    if (first < 0.0) first = fabs(a);
    if (!(fabs(a) > kMoveRatio * first)) break;
    for (int t = tid; t < nl; t += kCT) {
      const int i = lst[t];
      colp[i] = (double)__ldcg(X + i + (int64_t)p * r);
    }
    __syncthreads();
    if (tid == 0) {                           // remove p from the list
      const int tp = pos[p], last = lst[nl - 1];
      lst[tp] = last;
      pos[last] = tp;
      s_nl = nl - 1;
    }
    __syncthreads();
    const int m = nl - 1;
    const int nown = (m - rank + CS - 1) / CS;
    for (int64_t idx = tid; idx < (int64_t)m * nown; idx += kCT) {
      const int i = lst[(int)(idx % m)];
      const int j = lst[rank + CS * (int)(idx / m)];
      const double xpj = (double)__ldcg(X + p + (int64_t)j * r);
      X[i + (int64_t)j * r] =
          (Real)((double)__ldcg(X + i + (int64_t)j * r) - colp[i] * xpj / a);
    }
    cl.sync();
  }
  if (rank == 0 && tid == 0) {
    const int nl = s_nl;
    int c = 0;
    for (int i = 0; i < r; ++i)
      if (pos[i] < nl && lst[pos[i]] == i) ipool[D.piv_off + c++] = i;
    moves[q] = c;
  }
  cl.sync();  // no CTA leaves while another may still run
}

template <class Real>
cudaError_t launch_xrr_split_cluster(const LvlBox *lb, const int32_t *sel,
                                     int nsel, const int32_t *iscr,
                                     const Real *dscr, DevBox *boxes,
                                     Real *fac, int32_t *ipool,
                                     int32_t *moves, int max_n,
                                     cudaStream_t s) {
  if (nsel == 0) return cudaSuccess;
  size_t smem = (size_t)max_n * 20 + 64;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  void *args[] = {(void *)&lb,    (void *)&sel,   (void *)&iscr,
                  (void *)&dscr,  (void *)&boxes, (void *)&fac,
                  (void *)&ipool, (void *)&moves};
  cudaError_t e = launch_cluster((const void *)k_xrr_split_cluster<kCS, Real>,
                                 nsel, smem, s, args, kCS);
  note_launches(1);
  return e;
}

#define SKEL_INST(R)                                                           \
  template cudaError_t launch_cpqr_cluster<R, R>(                              \
      const LvlBox *, const int32_t *, int, int32_t *, R *, DevBox *, R *,     \
      double *, double, int, int, cudaStream_t, int);                          \
  template cudaError_t launch_eliminate_cluster<R>(                            \
      const LvlBox *, const int32_t *, int, const int32_t *, const R *,        \
      DevBox *, R *, int32_t *, int32_t *, int, int *, int, int32_t *,         \
      cudaStream_t, int);                                                      \
  template cudaError_t launch_xrr_split_cluster<R>(                            \
      const LvlBox *, const int32_t *, int, const int32_t *, const R *,        \
      DevBox *, R *, int32_t *, int32_t *, int, cudaStream_t);
SKEL_INST(double)
SKEL_INST(float)
#undef SKEL_INST
// FP32 ID matrix with FP64 factors
template cudaError_t launch_cpqr_cluster<float, double>(
    const LvlBox *, const int32_t *, int, int32_t *, float *, DevBox *,
    double *, double *, double, int, int, cudaStream_t, int);

}  // namespace skel
