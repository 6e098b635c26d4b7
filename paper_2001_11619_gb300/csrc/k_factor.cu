// Per-level box compression kernels, one CTA per box, for the FP64 form
// (Real = double) and the mixed form (Real = float):
//   * diagonal block of every box at the start of its level (Eq.
//     levelcompress: children's X_SS on the diagonal, original entries of
//     -1/2 I + D + N between siblings);
//   * the proxy ID matrix of Sec. 2.5 (Eq. gammaT) with both sides of the
//     nonsymmetric kernel (Sec. 2.4) and the two rows of the far part of the
//     rank-one completion N;
//   * column-pivoted Householder QR to a relative tolerance and
//     T = R11^{-1} R12 (Sec. 2.2), the triangular solve always in FP64;
//   * elimination of the redundant DOFs: Eq. (tmat) then the block LU of
//     Eq. (schurmat), giving LU(X_RR), Y = X_RR^{-1} X_RS,
//     Z = X_SR X_RR^{-1} and the Schur complement X_SS.
#include "qr_util.cuh"
#include "reduce.cuh"

namespace skel {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxProxy = 256;
// rows per lane per load batch in the one-CTA CPQR's reflector application:
// 8 for float storage (fewer dependent L2 round trips per step), 4 for the
// FP64 form (bound by the FP64 pipe; deeper batches only add registers)
template <class Real> struct CpqrReflect {
  static constexpr int RB = sizeof(Real) == 4 ? 8 : 4;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum and argmax over kWarps warps (reduce.cuh): every thread
// receives the result; scratch arrays hold kWarps + 1 entries.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
  return block_sum_w0<kWarps>(v, scratch);
}

// ties go to the lowest index
__device__ __forceinline__ void block_argmax(double &v, int &idx,
                                             long long *sk, int *si) {
  block_amax<kWarps>(v, idx, sk, si);
}

// ---------------------------------------------------------------------------
// diagonal block (n x n, column-major) of one box: entries of type Out,
// children's Schur complements stored as Real

// Entries idx0, idx0 + step, ... of the block (column-major order).
template <class Real, class Out>
__device__ void diag_block(const DevGeom &g, const LvlBox &B,
                           const int32_t *act, const Real *fac, Out *out,
                           int64_t ld, int64_t idx0, int64_t step) {
  const int n = B.n;
  for (int64_t idx = idx0; idx < (int64_t)n * n; idx += step) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    int ci = -1, cj = -1;
    for (int c = 0; c < B.nchild; ++c) {
      if (i >= B.cseg[c] && i < B.cseg[c] + B.ck[c]) ci = c;
      if (j >= B.cseg[c] && j < B.cseg[c] + B.ck[c]) cj = c;
    }
    Out v;
    if (ci >= 0 && ci == cj) {
      const int kc = B.ck[ci];
      v = (Out)fac[B.cxss[ci] + (i - B.cseg[ci]) +
                   (int64_t)(j - B.cseg[ci]) * kc];
    } else {
      v = a11_entry_r<Out>(g, act[i], act[j]);
    }
    out[i + j * ld] = v;
  }
}

template <class Real>
__global__ void k_assemble_diag(DevGeom g, const LvlBox *lb,
                                const int32_t *iscr, Real *dscr,
                                const Real *fac) {
  // grid: x = box, y = slice of its entries
  const LvlBox &B = lb[blockIdx.x];
  diag_block<Real, Real>(g, B, iscr + B.act_off, fac, dscr + B.a_off, B.n,
                         (int64_t)blockIdx.y * blockDim.x + threadIdx.x,
                         (int64_t)gridDim.y * blockDim.x);
}

// CTAs per box for the assembly kernels: levels with few (large) boxes
// spread each box over many CTAs, so that a level fills the GPU.
static int assembly_split(int nbox) {
  return std::max(1, std::min(256, (8 * 152 + nbox - 1) / nbox));
}

template <class Real>
void launch_assemble_diag(const DevGeom &g, const LvlBox *lb, int nbox,
                          const int32_t *iscr, Real *dscr, const Real *fac,
                          cudaStream_t s) {
  if (nbox == 0) return;
  dim3 grid(nbox, assembly_split(nbox));
  k_assemble_diag<Real><<<grid, kThreads, 0, s>>>(g, lb, iscr, dscr, fac);
  note_launches(1);
}

// the root block is always assembled in FP64 into the top matrix
template <class Real>
__global__ void k_root_block(DevGeom g, const LvlBox *lb, const int32_t *iscr,
                             const Real *fac, double *top, int ld) {
  const LvlBox &B = lb[0];
  diag_block<Real, double>(g, B, iscr + B.act_off, fac, top, ld,
                           (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                           (int64_t)gridDim.x * blockDim.x);
}

template <class Real>
void launch_root_block(const DevGeom &g, const LvlBox *lb, const int32_t *iscr,
                       const Real *fac, double *top, int ld, cudaStream_t s) {
  k_root_block<Real><<<2 * 152, kThreads, 0, s>>>(g, lb, iscr, fac, top, ld);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// proxy ID matrix (m x n, column-major, ld m).  Row blocks:
//   [0, nf)            K_{F_int,B}
//   [nf, nf+2P)        K_{P,B}: double layer from B to proxy point k,
//                      component c at row nf + c P + k
//   [nf+2P, 2nf+2P)    (K_{B,F_int})^T
//   [2nf+2P, 2nf+4P)   Stokeslet sources on the ring: G(x_B - p_k) wbar_B
//   [2nf+4P, 2nf+6P)   double-layer sources on the ring: D(x_B, p_k) wbar_B
//   2nf+6P, 2nf+6P+1   (w n)_B and wbar_B n_B (far part of N)

struct ProxyTab {
  double px[kMaxProxy], py[kMaxProxy], c[kMaxProxy], s[kMaxProxy];
  float pxh[kMaxProxy], pxl[kMaxProxy], pyh[kMaxProxy], pyl[kMaxProxy];
};

// block (a, b) of the proxy-row kernels for node j and ring point k:
// kind 0: D(p_k, x_j) w_j   kind 1: G(x_j - p_k) wp   kind 2: D(x_j, p_k) wp
__device__ __forceinline__ double proxy_entry_d(const DevGeom &g,
                                                const ProxyTab &pt, int kind,
                                                int j, int k, double wp,
                                                int a, int b) {
  double d00, d01, d11;
  if (kind == 0) {
    dl_block(pt.px[k], pt.py[k], g.x[j], g.y[j], g.nx[j], g.ny[j], g.w[j],
             d00, d01, d11);
  } else if (kind == 1) {
    stokeslet(g.x[j] - pt.px[k], g.y[j] - pt.py[k], d00, d01, d11);
    d00 *= wp;
    d01 *= wp;
    d11 *= wp;
  } else {
    dl_block(g.x[j], g.y[j], pt.px[k], pt.py[k], pt.c[k], pt.s[k], wp, d00,
             d01, d11);
  }
  return pick(d00, d01, d11, a, b);
}

__device__ __forceinline__ float proxy_entry_f(const DevGeom &g,
                                               const ProxyTab &pt, int kind,
                                               int j, int k, float wp, int a,
                                               int b) {
  // r = x_j - p_k from the float pairs
  const float rx = (g.xh[j] - pt.pxh[k]) + (g.xl[j] - pt.pxl[k]);
  const float ry = (g.yh[j] - pt.pyh[k]) + (g.yl[j] - pt.pyl[k]);
  float d00, d01, d11;
  if (kind == 0) {
    dl_block_f(-rx, -ry, g.nxf[j], g.nyf[j], g.wf[j], d00, d01, d11);
  } else if (kind == 1) {
    stokeslet_f(rx, ry, d00, d01, d11);
    d00 *= wp;
    d01 *= wp;
    d11 *= wp;
  } else {
    dl_block_f(rx, ry, (float)pt.c[k], (float)pt.s[k], wp, d00, d01, d11);
  }
  return pick(d00, d01, d11, a, b);
}

template <class Real>
__device__ __forceinline__ Real proxy_entry(const DevGeom &g,
                                            const ProxyTab &pt, int kind,
                                            int j, int k, double wp, int a,
                                            int b);
template <>
__device__ __forceinline__ double proxy_entry<double>(
    const DevGeom &g, const ProxyTab &pt, int kind, int j, int k, double wp,
    int a, int b) {
  return proxy_entry_d(g, pt, kind, j, k, wp, a, b);
}
template <>
__device__ __forceinline__ float proxy_entry<float>(
    const DevGeom &g, const ProxyTab &pt, int kind, int j, int k, double wp,
    int a, int b) {
  return proxy_entry_f(g, pt, kind, j, k, (float)wp, a, b);
}

template <class Real>
__global__ void __launch_bounds__(kThreads) k_assemble_id(DevGeom g, const LvlBox *lb, const int32_t *iscr,
                              Real *dscr, int P) {
  __shared__ double scratch[kWarps + 1];
  __shared__ ProxyTab pt;
  const LvlBox &B = lb[blockIdx.x];
  const int32_t *act = iscr + B.act_off;
  const int32_t *fint = iscr + B.fint_off;
  Real *M = dscr + B.m_off;
  const int n = B.n, m = B.m, nf = B.nf;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * k / P, &sn, &cs);
    const double px = B.cx + B.rho * cs, py = B.cy + B.rho * sn;
    pt.px[k] = px;
    pt.py[k] = py;
    pt.c[k] = cs;
    pt.s[k] = sn;
    const float pxh = (float)px, pyh = (float)py;
    pt.pxh[k] = pxh;
    pt.pxl[k] = (float)(px - (double)pxh);
    pt.pyh[k] = pyh;
    pt.pyl[k] = (float)(py - (double)pyh);
  }
  double ws = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    ws += g.w[g.lap ? act[i] : act[i] >> 1];  // node of the DOF
  // wbar: mean node weight of the box's active DOFs.  The ring sources
  // stand in for far rows (K_{B,F})^T whose entries carry the far nodes'
  // weights, so they are weighted by wbar (not by the ring's quadrature
  // weight 2 pi rho / P, which would make them dominate the relative ID
  // tolerance more and more as the discretization is refined).
  const double wbar = n > 0 ? block_sum(ws, scratch) / n : 0.0;
  const int64_t step = (int64_t)gridDim.y * blockDim.x;
  if (g.lap) {
    // Laplace form, one DOF per node; m = 2 nf + 4P + 2 rows:
    //   D(near targets <- B)            nf
    //   grad G(ring <- B) w_B           2P  (far targets, any normal)
    //   D(B <- near sources)            nf
    //   D(B <- ring charges) wbar,
    //   dn_x dn_p G(B <- ring dipoles) wbar   2P  (far sources)
    //   N: w_B and wbar 1               2
    for (int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
         idx < (int64_t)m * n; idx += step) {
      const int row = (int)(idx % m), col = (int)(idx / m);
      const int jc = act[col];
      double v;
      if (row < nf) {
        v = lap_d_entry(g, fint[row], jc);
      } else if (row < nf + 2 * P) {
        const int q = row - nf, c = q / P, pk = q % P;
        const double rx = pt.px[pk] - g.x[jc], ry = pt.py[pk] - g.y[jc];
        v = -(c ? ry : rx) / (2.0 * kPi * (rx * rx + ry * ry)) * g.w[jc];
      } else if (row < 2 * nf + 2 * P) {
        v = lap_d_entry(g, jc, fint[row - nf - 2 * P]);
      } else if (row < 2 * nf + 4 * P) {
        const int q = row - 2 * nf - 2 * P, blk = q / P, pk = q % P;
        const double rx = g.x[jc] - pt.px[pk], ry = g.y[jc] - pt.py[pk];
        const double inv = 1.0 / (rx * rx + ry * ry);
        const double rnx = rx * g.nx[jc] + ry * g.ny[jc];
        if (blk == 0) {
          v = -rnx * inv / (2.0 * kPi);
        } else {
          const double rnp = rx * pt.c[pk] + ry * pt.s[pk];
          const double nn = g.nx[jc] * pt.c[pk] + g.ny[jc] * pt.s[pk];
          v = (nn * inv - 2.0 * rnp * rnx * inv * inv) / (2.0 * kPi);
        }
        v *= wbar;
      } else {
        v = row == 2 * nf + 4 * P ? g.w[jc] : wbar;
      }
      M[idx] = (Real)v;
    }
    return;
  }
  for (int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
       idx < (int64_t)m * n; idx += step) {
    const int row = (int)(idx % m), col = (int)(idx / m);
    const int dc = act[col];
    const int jc = dc >> 1, bc = dc & 1;
    Real v;
    if (row < nf) {
      v = k_entry_r<Real>(g, fint[row], dc);
    } else if (row < nf + 2 * P) {
      const int q = row - nf, c = q / P, pk = q % P;
      v = proxy_entry<Real>(g, pt, 0, jc, pk, 0.0, c, bc);  // uses w_j
    } else if (row < 2 * nf + 2 * P) {
      v = k_entry_r<Real>(g, dc, fint[row - nf - 2 * P]);
    } else if (row < 2 * nf + 6 * P) {
      int q = row - 2 * nf - 2 * P;
      const int blk = q / (2 * P);
      q %= 2 * P;
      const int c = q / P, pk = q % P;
      v = proxy_entry<Real>(g, pt, 1 + blk, jc, pk, wbar, bc, c);
    } else {
      const double nv = bc ? g.ny[jc] : g.nx[jc];
      v = (Real)((row == 2 * nf + 6 * P) ? g.w[jc] * nv : wbar * nv);
    }
    M[idx] = v;
  }
}

template <class Real>
void launch_assemble_id(const DevGeom &g, const LvlBox *lb, int nbox,
                        const int32_t *iscr, Real *dscr, int n_proxy,
                        cudaStream_t s) {
  if (nbox == 0) return;
  // grid: x = box, y = slice of its entries (each CTA also forms the box's
  // proxy table and mean weight, identically)
  dim3 grid(nbox, assembly_split(nbox));
  k_assemble_id<Real><<<grid, kThreads, 0, s>>>(g, lb, iscr, dscr, n_proxy);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// column-pivoted Householder QR with early stop, then T = R11^{-1} R12.
// Pivot norms are downdated with the LAPACK cancellation safeguard; the
// chosen pivot's norm is recomputed exactly (in FP64) before its reflector
// is formed and the stopping test is applied.  The ID matrix is stored as
// Real; T is solved in FP64 in the box's workspace tws and then stored in
// the factor type Fac.

// CTA size of the one-CTA CPQR (a box per CTA)
constexpr int kQT = 512;
constexpr int kQW = kQT / 32;

template <class Real, class Fac>
__global__ void __launch_bounds__(kQT) k_cpqr(const LvlBox *lb, const int32_t *sel, int32_t *iscr,
                       Real *dscr, DevBox *boxes, Fac *fac, double *tws,
                       double tol) {
  extern __shared__ double smem[];
  __shared__ double sv[kQW + 1];
  __shared__ double ss[3];  // this step's norm, alpha and tau
  __shared__ long long sk[kQW + 1];
  __shared__ int si[kQW + 1];
  const LvlBox &B = lb[sel[blockIdx.x]];
  const int n = B.n, m = B.m;
  Real *A = dscr + B.m_off;
  double *cn = smem;
  double *cn0 = smem + n;
  int *perm = (int *)(smem + 2 * n);
  Real *rj = (Real *)(perm + n + (n & 1));     // new row-j entries
  unsigned char *flag = (unsigned char *)(rj + n);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int c = warp; c < n; c += kQW) {
    Real sp = Real(0);  // per-lane partial sums in the storage type
    for (int i = lane; i < m; i += 32) {
      const Real a = A[i + (int64_t)c * m];
      sp += a * a;
    }
    const double s = (double)warp_sum_t<Real>(sp);
    if (lane == 0) {
      cn[c] = s;
      cn0[c] = s;
    }
  }
  for (int c = tid; c < n; c += kQT) perm[c] = c;
  __syncthreads();

  const int kmax = m < n ? m : n;
  int k = kmax;
  double r11 = 0.0;
  for (int j = 0; j < kmax; ++j) {
    double bv = -1.0;
    int bi = n;
    for (int c = j + tid; c < n; c += kQT)
      if (cn[c] > bv) {
        bv = cn[c];
        bi = c;
      }
    // (every step ends with a barrier, so the argmax slots are free)
    block_amax<kQW, false>(bv, bi, sk, si);
    const int p = bi;
    if (p >= n) {  // no finite column norm left (NaN input): stop here
      k = j;
      break;
    }
    // exact norm of the pivot's trailing rows, summed while the pivot
    // column moves to position j: per-thread partial sums in the storage
    // type, warp sums in that type, the warp totals in FP64 by warp 0,
    // whose lane 0 then forms the reflector's scalars once (the FP64 pipe
    // is the scarce one: a square root and a division in every thread
    // would cost more than the step's downdates) and writes v0 over the
    // diagonal
    Real sp = Real(0);
    if (p != j) {
      for (int i = tid; i < m; i += kQT) {
        const Real t = A[i + (int64_t)j * m], u = A[i + (int64_t)p * m];
        A[i + (int64_t)j * m] = u;
        A[i + (int64_t)p * m] = t;
        if (i >= j) sp += u * u;
      }
    } else {
      for (int i = j + tid; i < m; i += kQT) {
        const Real a = A[i + (int64_t)j * m];
        sp += a * a;
      }
    }
    if (p != j && tid == 0) {
      int t = perm[j];
      perm[j] = perm[p];
      perm[p] = t;
      double tc = cn[j];
      cn[j] = cn[p];
      cn[p] = tc;
      tc = cn0[j];
      cn0[j] = cn0[p];
      cn0[p] = tc;
    }
    sp = warp_sum_t<Real>(sp);
    if (lane == 0) sv[warp] = (double)sp;
    __syncthreads();
    if (warp == 0) {
      double t = lane < kQW ? sv[lane] : 0.0;
      t = qr_warp_sum(t);
      if (lane == 0) {
        const double nrm = sqrt(t);
        const double x0 = (double)A[j + (int64_t)j * m];
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        ss[0] = nrm;
        ss[1] = alpha;
        ss[2] = nrm > 0.0 ? 2.0 / (t - x0 * x0 + v0 * v0) : 0.0;
        const double r11j = j == 0 ? nrm : r11;
        if (!(nrm == 0.0 || nrm <= tol * r11j))  // the stopping test below
          A[j + (int64_t)j * m] = (Real)v0;
      }
    }
    __syncthreads();
    const double nrm = ss[0];
    if (j == 0) r11 = nrm;
    if (nrm == 0.0 || nrm <= tol * r11) {
      k = j;
      break;
    }
    const double alpha = ss[1], tau = ss[2];
    auto colq = [&](int q) { return j + 1 + q; };
    auto none = [](int) { return false; };
    apply_reflector<4, CpqrReflect<Real>::RB, Real, decltype(colq),
                    decltype(none), false>(
        A, m, j, A + (int64_t)j * m, tau, n - j - 1, colq, none,
        cn + j + 1, cn0 + j + 1, rj, flag, warp, kQW, lane);
    // every read of v (column j) ended before the reflector's downdate
    // barrier; the barrier below publishes alpha and the recomputed norms
    if (tid == 0) A[j + (int64_t)j * m] = (Real)alpha;
    __syncthreads();
  }
  __syncthreads();
  // T = R11^{-1} R12 in FP64: copy R12 to the workspace, then column-
  // oriented back substitution (R11 read from A and widened), multiplying
  // by the reciprocals of R11's diagonal (one division each, in parallel;
  // they replace the column norms in shared memory)
  const int r = n - k;
  double *W = tws + B.t_off;
  for (int64_t idx = tid; idx < (int64_t)k * r; idx += kQT) {
    const int i = (int)(idx % k), c = (int)(idx / k);
    W[idx] = (double)A[i + (int64_t)(k + c) * m];
  }
  for (int i = tid; i < k; i += kQT)
    cn[i] = 1.0 / (double)A[i + (int64_t)i * m];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double d = cn[i];
    for (int c = tid; c < r; c += kQT) W[i + (int64_t)c * k] *= d;
    __syncthreads();
    for (int64_t idx = tid; idx < (int64_t)i * r; idx += kQT) {
      const int l = (int)(idx % i), c = (int)(idx / i);
      W[l + (int64_t)c * k] -=
          (double)A[l + (int64_t)i * m] * W[i + (int64_t)c * k];
    }
    __syncthreads();
  }
  DevBox &D = boxes[B.box];
  Fac *T = fac + D.fac_off + fac_T(k, r);
  for (int64_t idx = tid; idx < (int64_t)k * r; idx += kQT)
    T[idx] = (Fac)W[idx];
  int32_t *po = iscr + B.perm_off;
  for (int c = tid; c < n; c += kQT) po[c] = perm[c];
  if (tid == 0) D.k = k;
}

template <class Real, class Fac>
void launch_cpqr(const LvlBox *lb, const int32_t *sel, int nbox,
                 int32_t *iscr, Real *dscr, DevBox *boxes, Fac *fac,
                 double *tws, double tol, int max_n, cudaStream_t s) {
  if (nbox == 0) return;
  const size_t sm = (size_t)max_n * (2 * sizeof(double) + sizeof(int) +
                                     sizeof(Real) + 1) + 64;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_cpqr<Real, Fac>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  // the rest of the SM's 256 KB as L1: the reflector's update pass re-reads
  // the columns its dot pass has just loaded
  cudaFuncSetAttribute(k_cpqr<Real, Fac>,
                       cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxL1);
  k_cpqr<Real, Fac><<<nbox, kQT, sm, s>>>(lb, sel, iscr, dscr, boxes, fac,
                                               tws, tol);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// elimination of the redundant DOFs of one box (all in Real)

template <class Real>
__global__ void __launch_bounds__(kThreads) k_eliminate(const LvlBox *lb, const int32_t *sel,
                            const int32_t *iscr, const Real *dscr,
                            DevBox *boxes, Real *fac, int32_t *ipool,
                            int32_t *dofs, int *status, int allow_move,
                            int32_t *flag) {
  extern __shared__ int sperm[];
  __shared__ double sv[kWarps + 1];
  __shared__ long long sk[kWarps + 1];
  __shared__ int si[kWarps + 1];
  const LvlBox &B = lb[sel[blockIdx.x]];
  DevBox &D = boxes[B.box];
  const int n = B.n, k = D.k, r = n - k;
  const int tid = threadIdx.x;
  const Real *A = dscr + B.a_off;
  const int32_t *act = iscr + B.act_off;
  const int32_t *perm_g = iscr + B.perm_off;
  for (int i = tid; i < n; i += kThreads) {
    sperm[i] = perm_g[i];
    dofs[D.dof_off + i] = act[perm_g[i]];
  }
  __syncthreads();
  const int *pm = sperm;
#define KA(i, j) A[pm[i] + (int64_t)pm[j] * n]
  Real *F = fac + D.fac_off;
  const Real *T = F + fac_T(k, r);
  Real *Y = F + fac_Y(k, r);
  Real *Z = F + fac_Z(k, r);
  Real *LU = F + fac_LU(k, r);
  Real *XSS = F + fac_XSS(k, r);
  int32_t *piv = ipool + D.piv_off;

  // Eq. (tmat): X_RS = K_RS - T^T K_SS  (r x k, into Y)
  for (int64_t idx = tid; idx < (int64_t)r * k; idx += kThreads) {
    const int i = (int)(idx % r), s = (int)(idx / r);
    Real acc = KA(k + i, s);
    for (int t = 0; t < k; ++t) acc -= T[t + (int64_t)i * k] * KA(t, s);
    Y[idx] = acc;
  }
  //             X_SR = K_SR - K_SS T  (k x r, into Z)
  for (int64_t idx = tid; idx < (int64_t)k * r; idx += kThreads) {
    const int s = (int)(idx % k), i = (int)(idx / k);
    Real acc = KA(s, k + i);
    for (int t = 0; t < k; ++t) acc -= KA(s, t) * T[t + (int64_t)i * k];
    Z[idx] = acc;
  }
  __syncthreads();
  //             X_RR = K_RR - T^T K_SR - X_RS T  (r x r, into LU)
  for (int64_t idx = tid; idx < (int64_t)r * r; idx += kThreads) {
    const int i = (int)(idx % r), j = (int)(idx / r);
    Real acc = KA(k + i, k + j);
    for (int t = 0; t < k; ++t)
      acc -= T[t + (int64_t)i * k] * KA(t, k + j) +
             Y[i + (int64_t)t * r] * T[t + (int64_t)j * k];
    LU[idx] = acc;
  }
  __syncthreads();
#undef KA
  // LU of X_RR with partial pivoting (LAPACK convention: whole rows swapped)
  double umax = 0.0, umin = INFINITY;
  for (int j = 0; j < r; ++j) {
    double bv = -1.0;
    int bi = r;
    for (int i = j + tid; i < r; i += kThreads) {
      const double a = fabs((double)LU[i + (int64_t)j * r]);
      if (a > bv) {
        bv = a;
        bi = i;
      }
    }
    block_argmax(bv, bi, sk, si);
    int p = bi;
    if (p >= r) {  // NaN column: keep the row order, flag the box singular
      p = j;
      bv = 0.0;
    }
    umax = fmax(umax, bv);
    umin = fmin(umin, bv);
    if (p != j)
      for (int c = tid; c < r; c += kThreads) {
        Real t = LU[j + (int64_t)c * r];
        LU[j + (int64_t)c * r] = LU[p + (int64_t)c * r];
        LU[p + (int64_t)c * r] = t;
      }
    if (tid == 0) piv[j] = p;
    __syncthreads();
    const Real d = LU[j + (int64_t)j * r];
    if (d != Real(0))
      for (int i = j + 1 + tid; i < r; i += kThreads) LU[i + (int64_t)j * r] /= d;
    __syncthreads();
    const int w = r - j - 1;
    for (int64_t idx = tid; idx < (int64_t)w * w; idx += kThreads) {
      const int i = j + 1 + (int)(idx % w), c = j + 1 + (int)(idx / w);
      LU[i + (int64_t)c * r] -= LU[i + (int64_t)j * r] * LU[j + (int64_t)c * r];
    }
    __syncthreads();
  }
  // X_RR conditioning (Sec. 2.2 remark): a pivot at or below kMoveRatio of
  // the largest flags the box and stops here (X_RS is still in Y); the
  // host then moves indices from R into S and eliminates it again.
  const bool moving = allow_move && r > 0 && !(umin > kMoveRatio * umax);
  if (tid == 0) flag[sel[blockIdx.x]] = moving ? 1 : 0;
  if (moving) return;
  if (r > 0 && tid == 0 && !(umin > 1e-14 * umax)) atomicMin(status, SKEL_ESINGULAR);
  // Y = X_RR^{-1} X_RS: row interchanges, unit-lower then upper solves
  for (int s = tid; s < k; s += kThreads)
    for (int j = 0; j < r; ++j) {
      const int p = piv[j];
      if (p != j) {
        Real t = Y[j + (int64_t)s * r];
        Y[j + (int64_t)s * r] = Y[p + (int64_t)s * r];
        Y[p + (int64_t)s * r] = t;
      }
    }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const int w = r - j - 1;
    for (int64_t idx = tid; idx < (int64_t)w * k; idx += kThreads) {
      const int i = j + 1 + (int)(idx % w), s = (int)(idx / w);
      Y[i + (int64_t)s * r] -= LU[i + (int64_t)j * r] * Y[j + (int64_t)s * r];
    }
    __syncthreads();
  }
  for (int j = r - 1; j >= 0; --j) {
    const Real d = LU[j + (int64_t)j * r];
    for (int s = tid; s < k; s += kThreads) Y[j + (int64_t)s * r] /= d;
    __syncthreads();
    for (int64_t idx = tid; idx < (int64_t)j * k; idx += kThreads) {
      const int i = (int)(idx % j), s = (int)(idx / j);
      Y[i + (int64_t)s * r] -= LU[i + (int64_t)j * r] * Y[j + (int64_t)s * r];
    }
    __syncthreads();
  }
  // Eq. (schurmat): X_SS = K_SS - X_SR Y (X_SR still held in Z)
  for (int64_t idx = tid; idx < (int64_t)k * k; idx += kThreads) {
    const int s = (int)(idx % k), t = (int)(idx / k);
    Real acc = A[sperm[s] + (int64_t)sperm[t] * n];
    for (int i = 0; i < r; ++i) acc -= Z[s + (int64_t)i * k] * Y[i + (int64_t)t * r];
    XSS[idx] = acc;
  }
  __syncthreads();
  // Z = X_SR X_RR^{-1}: with X_RR = P^T L U solve V U = X_SR, W L = V,
  // then Z = W P (column interchanges in reverse order)
  for (int j = 0; j < r; ++j) {
    const Real d = LU[j + (int64_t)j * r];
    for (int s = tid; s < k; s += kThreads) Z[s + (int64_t)j * k] /= d;
    __syncthreads();
    const int w = r - j - 1;
    for (int64_t idx = tid; idx < (int64_t)w * k; idx += kThreads) {
      const int s = (int)(idx % k), c = j + 1 + (int)(idx / k);
      Z[s + (int64_t)c * k] -= Z[s + (int64_t)j * k] * LU[j + (int64_t)c * r];
    }
    __syncthreads();
  }
  for (int j = r - 1; j >= 0; --j) {
    for (int64_t idx = tid; idx < (int64_t)j * k; idx += kThreads) {
      const int s = (int)(idx % k), c = (int)(idx / k);
      Z[s + (int64_t)c * k] -= Z[s + (int64_t)j * k] * LU[j + (int64_t)c * r];
    }
    __syncthreads();
  }
  for (int s = tid; s < k; s += kThreads)
    for (int j = r - 1; j >= 0; --j) {
      const int p = piv[j];
      if (p != j) {
        Real t = Z[s + (int64_t)j * k];
        Z[s + (int64_t)j * k] = Z[s + (int64_t)p * k];
        Z[s + (int64_t)p * k] = t;
      }
    }
}

template <class Real>
void launch_eliminate(const LvlBox *lb, const int32_t *sel, int nbox,
                      const int32_t *iscr, const Real *dscr, DevBox *boxes,
                      Real *fac, int32_t *ipool, int32_t *dofs, int max_n,
                      int *status, int allow_move, int32_t *flag,
                      cudaStream_t s) {
  if (nbox == 0) return;
  const size_t sm = (size_t)max_n * sizeof(int) + 16;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_eliminate<Real>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eliminate<Real><<<nbox, kThreads, sm, s>>>(lb, sel, iscr, dscr, boxes, fac,
                                               ipool, dofs, status, allow_move,
                                               flag);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// Moving redundant indices into the skeleton (Sec. 2.2 remark).  For box q
// with cnt = moves[q] > 0, the positions J (ascending, counted inside the
// redundant block) sit in the box's pivot slot of ipool.  The new partition
// is S' = S + J, R' = R - J: the permutation becomes [S, R_J, R_kept] and
// T' = [T restricted to the kept columns; zero rows for J] (k' x r', ld
// k'), so K_{F,R'} ~ K_{F,S'} T' still holds and X_{R'R'} is a principal
// block of X_RR.  T' goes to the FP64 workspace (through its second half)
// and to the factor slot; D.k becomes k'.
template <class Fac>
__global__ void __launch_bounds__(kThreads) k_repartition(const LvlBox *lb, const int32_t *sel,
                              int32_t *iscr, DevBox *boxes, Fac *fac,
                              const int32_t *ipool, const int32_t *moves,
                              double *tws, int64_t tws_half) {
  extern __shared__ int shp[];
  const int q = sel[blockIdx.x];
  const LvlBox &B = lb[q];
  DevBox &D = boxes[B.box];
  const int n = B.n, k = D.k, r = n - k;
  const int cnt = moves[q];
  const int k2 = k + cnt, r2 = r - cnt;
  int *nperm = shp;        // n
  int *keep = shp + n;     // r2
  const int32_t *J = ipool + D.piv_off;
  int32_t *perm = iscr + B.perm_off;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int jn = 0, kn = 0;
    for (int i = 0; i < r; ++i) {
      if (jn < cnt && J[jn] == i) {
        nperm[k + jn] = perm[k + i];
        ++jn;
      } else {
        keep[kn] = i;
        nperm[k2 + kn] = perm[k + i];
        ++kn;
      }
    }
  }
  for (int i = tid; i < k; i += blockDim.x) nperm[i] = perm[i];
  __syncthreads();
  const double *T = tws + B.t_off;
  double *T2 = tws + tws_half + B.t_off;
  for (int64_t idx = tid; idx < (int64_t)k2 * r2; idx += blockDim.x) {
    const int i = (int)(idx % k2), c = (int)(idx / k2);
    T2[idx] = i < k ? T[i + (int64_t)keep[c] * k] : 0.0;
  }
  __syncthreads();
  double *Tw = tws + B.t_off;
  Fac *Tf = fac + D.fac_off + fac_T(k2, r2);
  for (int64_t idx = tid; idx < (int64_t)k2 * r2; idx += blockDim.x) {
    const double v = T2[idx];
    Tw[idx] = v;
    Tf[idx] = (Fac)v;
  }
  for (int i = tid; i < n; i += blockDim.x) perm[i] = nperm[i];
  if (tid == 0) D.k = k2;
}

template <class Fac>
void launch_repartition(const LvlBox *lb, const int32_t *sel, int nbox,
                        int32_t *iscr, DevBox *boxes, Fac *fac,
                        const int32_t *ipool, const int32_t *moves,
                        double *tws, int64_t tws_half, int max_n,
                        cudaStream_t s) {
  if (nbox == 0) return;
  const size_t sm = (size_t)2 * max_n * sizeof(int) + 16;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_repartition<Fac>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_repartition<Fac><<<nbox, kThreads, sm, s>>>(lb, sel, iscr, boxes, fac,
                                                ipool, moves, tws, tws_half);
  note_launches(1);
}

// explicit instantiations for both forms
#define SKEL_INST(R)                                                          \
  template void launch_assemble_diag<R>(const DevGeom &, const LvlBox *, int, \
                                        const int32_t *, R *, const R *,      \
                                        cudaStream_t);                        \
  template void launch_root_block<R>(const DevGeom &, const LvlBox *,         \
                                     const int32_t *, const R *, double *,    \
                                     int, cudaStream_t);                      \
  template void launch_assemble_id<R>(const DevGeom &, const LvlBox *, int,   \
                                      const int32_t *, R *, int,              \
                                      cudaStream_t);                          \
  template void launch_cpqr<R, R>(const LvlBox *, const int32_t *, int,       \
                                  int32_t *, R *, DevBox *, R *, double *,    \
                                  double, int, cudaStream_t);                 \
  template void launch_eliminate<R>(const LvlBox *, const int32_t *, int,     \
                                    const int32_t *, const R *, DevBox *,     \
                                    R *, int32_t *, int32_t *, int, int *,    \
                                    int, int32_t *, cudaStream_t);            \
  template void launch_repartition<R>(const LvlBox *, const int32_t *, int,   \
                                      int32_t *, DevBox *, R *,               \
                                      const int32_t *, const int32_t *,       \
                                      double *, int64_t, int, cudaStream_t);
SKEL_INST(double)
SKEL_INST(float)
#undef SKEL_INST
// FP32 ID matrix with FP64 factors
template void launch_cpqr<float, double>(const LvlBox *, const int32_t *, int,
                                         int32_t *, float *, DevBox *,
                                         double *, double *, double, int,
                                         cudaStream_t);

}  // namespace skel
