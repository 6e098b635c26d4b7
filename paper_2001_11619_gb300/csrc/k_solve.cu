// Factored solve kernels (Eq. kinv, Sec. 2.7 last paragraph, Sec. 3.2):
//   * level sweeps applying U / V (and V^T / U^T for the adjoint) box by
//     box, every box of a level on disjoint DOFs, one CTA per box;
//   * the bordered top block of Eq. (partition) and its dense LU;
//   * masked reductions over the redundant rows for the coupling terms.
// All FP64.
#include "kmath.cuh"
#include "reduce.cuh"
#include "wide_util.cuh"

namespace skel {

// ---------------------------------------------------------------------------
// out = A_R^T B_R over the rows with rmask set (A, B: rows x cols, ld).
//
// A is the bordered block Psi^T V (QT): its column a belongs to one hole,
// and V^T only mixes DOFs inside a box, so QT(j, a) is exactly zero unless
// the box that eliminates DOF j holds part of that hole in its subtree.  On
// the 1M-node, 256-hole case a column has about 10^4 nonzero rows out of
// 2 x 10^6.  The product therefore runs in two steps:
//   1. per column a, the ordered list of 32-row chunks with a nonzero
//      masked entry (one CTA per column, ballots and a block prefix sum);
//   2. per column a and 32 columns c of B, one CTA sums QT(j, a) B(j, c)
//      over the listed chunks, lane = row of the chunk, warps taking the
//      chunks in turn, then a fixed-order reduction over lanes and warps.
// Every sum has a fixed order (deterministic), and only the zero products
// of the masked-out and zero rows are skipped.
// top right-hand side and back substitution: slabs of kTS rows staged in
// shared memory against 32 border columns and up to kTQ right-hand sides
constexpr int kTS = 64;
constexpr int kTQ = 32;

size_t gram_scratch_ints(int64_t rows, int cols) {
  return (size_t)cols * ((rows + 31) / 32) + cols + 1;
}

__global__ void __launch_bounds__(256)
k_gram_chunklist(const double *A, int64_t rows, int64_t ld,
                 const uint8_t *rmask, int64_t nchunks, int32_t *list,
                 int32_t *cnt) {
  __shared__ int wsum[8];
  const int a = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double *Aa = A + ld * a;
  int32_t *out = list + (int64_t)a * nchunks;
  int64_t base = 0;
  for (int64_t c0 = 0; c0 < nchunks; c0 += 256) {
    int flag = 0;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const int64_t ch = c0 + 32 * w + i;
      const int64_t row = ch * 32 + lane;
      bool nz = false;
      if (ch < nchunks && row < rows) nz = rmask[row] && Aa[row] != 0.0;
      const unsigned b = __ballot_sync(0xffffffffu, nz);
      if (lane == i) flag = b != 0u;
    }
    const unsigned fb = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) wsum[w] = __popc(fb);
    __syncthreads();
    int64_t off = base;
    int tot = 0;
    for (int v = 0; v < 8; ++v) {
      if (v < w) off += wsum[v];
      tot += wsum[v];
    }
    if (flag) out[off + __popc(fb & ((1u << lane) - 1u))] =
        (int32_t)(c0 + 32 * w + lane);
    __syncthreads();
    base += tot;
  }
  if (threadIdx.x == 0) cnt[a] = (int32_t)base;
}

__global__ void __launch_bounds__(256)
k_gram_sparse(const double *A, const double *B, int64_t rows, int64_t ld,
              int cols, const uint8_t *rmask, const int32_t *list,
              int64_t nchunks, const int32_t *cnt, double *out) {
  __shared__ double sred[8][33];
  const int a = blockIdx.x, cb = blockIdx.y * 32;
  const int nc = cols - cb < 32 ? cols - cb : 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double *Aa = A + ld * a;
  const int32_t *L = list + (int64_t)a * nchunks;
  const int n = cnt[a];
  double acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.0;
  for (int t = w; t < n; t += 8) {
    const int64_t row = (int64_t)L[t] * 32 + lane;
    double qa = 0.0;
    if (row < rows && rmask[row]) qa = Aa[row];
    if (qa != 0.0) {
      const double *Br = B + row + ld * cb;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < nc) acc[c] += qa * Br[ld * c];
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sred[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double v = 0.0;
    for (int u = 0; u < 8; ++u) v += sred[u][threadIdx.x];
    out[a + (int64_t)(cb + threadIdx.x) * cols] = v;
  }
}

// Rows per CTA of the top right-hand side: whole slabs, and about 16 CTAs
// per SM over the (row chunk, column tile, right-hand-side tile) grid.
static int64_t top_rhs_rows(int64_t n2, int p3, int nrhs) {
  const int64_t tiles =
      (int64_t)((p3 + 31) / 32) * ((nrhs + kTQ - 1) / kTQ);
  const int64_t slabs = (n2 + kTS - 1) / kTS;
  int64_t want = (16 * 152 + tiles - 1) / tiles;
  if (want > slabs) want = slabs;
  if (want < 1) want = 1;
  return (slabs + want - 1) / want * kTS;
}

int top_rhs_chunks(int64_t n2, int p3, int nrhs) {
  if (n2 == 0) return 1;
  const int64_t rows = top_rhs_rows(n2, p3, nrhs);
  return (int)((n2 + rows - 1) / rows);
}

void launch_gram_masked(const double *A, const double *B, int64_t rows,
                        int64_t ld, int cols, const uint8_t *rmask,
                        int32_t *scratch, double *out, cudaStream_t s) {
  if (cols == 0) return;
  const int64_t nchunks = (rows + 31) / 32;
  int32_t *list = scratch, *cnt = scratch + (int64_t)cols * nchunks;
  k_gram_chunklist<<<cols, 256, 0, s>>>(A, rows, ld, rmask, nchunks, list,
                                        cnt);
  note_launches(1);
  dim3 grid((unsigned)cols, (unsigned)((cols + 31) / 32));
  k_gram_sparse<<<grid, 256, 0, s>>>(A, B, rows, ld, cols, rmask, list,
                                     nchunks, cnt, out);
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
// Blocked right-looking LU (LAPACK convention).  Per panel of kNB columns:
// the panel is factored by one CTA, its row interchanges are applied to the
// other columns together with the unit-lower solve for U12, and the
// trailing block is updated by a tiled FP64 GEMM over all SMs.
constexpr int kNB = 32;

__global__ void k_panel_lu(double *A, int n, int ld, int j0, int jb,
                           int32_t *piv, double *ustat, int32_t *map,
                           double *rdiag) {
  // the panel A[j0:n, j0:j0+jb] is factored in shared memory
  extern __shared__ double P[];
  __shared__ long long sk[33];
  __shared__ int si[33];
  __shared__ double s_rd;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rows = n - j0;
  for (int idx = tid; idx < rows * jb; idx += nt) {
    const int i = idx % rows, c = idx / rows;
    P[idx] = A[(j0 + i) + (int64_t)(j0 + c) * ld];
  }
  __syncthreads();
  // pivot candidates of column 0; later ones come out of the update
  double bv = -1.0;
  int bi = rows;
  for (int i = tid; i < rows; i += nt) {
    const double a = fabs(P[i]);
    if (a > bv) {
      bv = a;
      bi = i;
    }
  }
  for (int jj = 0; jj < jb; ++jj) {
    block_amax<32>(bv, bi, sk, si);  // launched with 1024 threads
    const int p = bi < rows ? bi : jj;  // NaN column: no interchange
    if (bi >= rows) bv = 0.0;
    const int col = j0 + jj;
    if (tid == 0) {
      piv[col] = j0 + p;
      ustat[0] = col == 0 ? bv : fmax(ustat[0], bv);
      ustat[1] = col == 0 ? bv : fmin(ustat[1], bv);
    }
    if (tid == jj) {
      // the reciprocal of the pivot, once, by the thread that moves it
      // (kept for the solves); the other threads wait at the barrier
      const double d = P[p + (int64_t)jj * rows];
      const double r = d != 0.0 ? 1.0 / d : 0.0;
      s_rd = r;
      rdiag[col] = r;
    }
    if (p != jj && tid < jb) {
      double t = P[jj + (int64_t)tid * rows];
      P[jj + (int64_t)tid * rows] = P[p + (int64_t)tid * rows];
      P[p + (int64_t)tid * rows] = t;
    }
    __syncthreads();
    // each thread's rows below the pivot: scale, the rank-one update of
    // the panel's later columns, and the next column's pivot candidate,
    // with no barrier in between
    const double rd = s_rd;
    double nbv = -1.0;
    int nbi = rows;
    for (int i = jj + 1 + tid; i < rows; i += nt) {
      double l = P[i + (int64_t)jj * rows];
      if (rd != 0.0) {
        l *= rd;
        P[i + (int64_t)jj * rows] = l;
      }
      for (int c = jj + 1; c < jb; ++c)
        P[i + (int64_t)c * rows] -= l * P[jj + (int64_t)c * rows];
      if (jj + 1 < jb) {
        const double a = fabs(P[i + (int64_t)(jj + 1) * rows]);
        if (a > nbv) {
          nbv = a;
          nbi = i;
        }
      }
    }
    bv = nbv;
    bi = nbi;
  }
  __syncthreads();
  for (int idx = tid; idx < rows * jb; idx += nt) {
    const int i = idx % rows, c = idx / rows;
    A[(j0 + i) + (int64_t)(j0 + c) * ld] = P[idx];
  }
  // the panel's interchanges composed into one row map for the other
  // columns: map[0] = count, then (row, source row) pairs, row <- source
  if (tid == 0) {
    int rows_t[2 * kNB], src_t[2 * kNB], cnt = 0;
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
    map[0] = cnt;
    for (int q = 0; q < cnt; ++q) {
      map[1 + 2 * q] = rows_t[q];
      map[2 + 2 * q] = src_t[q];
    }
  }
}

int lu_map_doubles() { return (1 + 4 * kNB) / 2 + 1; }

int lu_extra_doubles(int n) { return 2 + lu_map_doubles() + n; }

// reciprocals of U's diagonal, after the pivot statistics and the row map
static double *lu_rdiag(const double *A, int n, int ld) {
  return const_cast<double *>(A) + (int64_t)ld * n + 2 + lu_map_doubles();
}

// columns outside the panel, one warp per column: the panel's row map
// applied at once (every lane gathers its entries, then all write), then
// (right of the panel) U12 = L11^{-1} A12 with the unit-lower L11, the
// column's panel rows held one per lane and solved by shuffles
__global__ void k_lu_swap_trsm_w(double *A, int n, int ld, int j0, int jb,
                                 const int32_t *map) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int c = w < j0 ? w : w + jb;
  if (c >= n) return;  // whole warps
  double *col = A + (int64_t)c * ld;
  const int cnt = map[0];
  double v[2];
  int r[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    r[h] = q < cnt ? map[1 + 2 * q] : -1;
    v[h] = q < cnt ? col[map[2 + 2 * q]] : 0.0;
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (r[h] >= 0) col[r[h]] = v[h];
  __syncwarp();
  if (c < j0 + jb) return;
  double x = lane < jb ? col[j0 + lane] : 0.0;
  for (int jj = 0; jj < jb; ++jj) {
    const double xj = __shfl_sync(0xffffffffu, x, jj);
    if (lane > jj && lane < jb)
      x -= A[(j0 + lane) + (int64_t)(j0 + jj) * ld] * xj;
  }
  if (lane < jb) col[j0 + lane] = x;
}

// A22 -= L21 U12, 64x64 output tiles, 256 threads with 4x4 outputs each
__global__ void __launch_bounds__(256)
k_lu_gemm(double *A, int n, int ld, int j0, int jb) {
  __shared__ double Ls[kNB][64 + 1];
  __shared__ double Us[kNB][64 + 1];
  const int base = j0 + jb;
  const int r0 = base + blockIdx.x * 64, c0 = base + blockIdx.y * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int idx = threadIdx.x; idx < 64 * jb; idx += 256) {
    int i = idx % 64, kk = idx / 64;
    int r = r0 + i;
    Ls[kk][i] = r < n ? A[r + (int64_t)(j0 + kk) * ld] : 0.0;
    int c = c0 + i;
    Us[kk][i] = c < n ? A[(j0 + kk) + (int64_t)c * ld] : 0.0;
  }
  __syncthreads();
  double acc[4][4] = {};
  for (int kk = 0; kk < jb; ++kk) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Ls[kk][tx + 16 * u];
      b[u] = Us[kk][ty + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int r = r0 + tx + 16 * u, c = c0 + ty + 16 * v;
      if (r < n && c < n) A[r + (int64_t)c * ld] -= acc[u][v];
    }
}

int launch_dense_lu(double *A, int n, int ld, int32_t *piv, int *,
                    cudaStream_t s) {
  // ustat lives in the two doubles after the matrix, the panel row map
  // after them (caller allocates lu_map_doubles() more)
  double *ustat = A + (int64_t)ld * n;
  int32_t *map = reinterpret_cast<int32_t *>(ustat + 2);
  double *rdiag = lu_rdiag(A, n, ld);
  // panel width: the panel (n x nb doubles) must fit in shared memory
  int nb = kNB;
  while (nb > 1 && (size_t)n * nb * 8 > 200 * 1024) nb /= 2;
  const size_t psm = (size_t)n * nb * 8;
  if (psm > 48 * 1024)
    cudaFuncSetAttribute(k_panel_lu,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = n - j0 < nb ? n - j0 : nb;
    k_panel_lu<<<1, 1024, (size_t)(n - j0) * jb * 8, s>>>(A, n, ld, j0, jb,
                                                         piv, ustat, map,
                                                         rdiag);
    note_launches(1);
    const int others = n - jb;
    if (others > 0) {
      k_lu_swap_trsm_w<<<(others + 7) / 8, 256, 0, s>>>(A, n, ld, j0, jb,
                                                        map);
      note_launches(1);
    }
    const int rest = n - j0 - jb;
    if (rest > 0) {
      dim3 grid((rest + 63) / 64, (rest + 63) / 64);
      k_lu_gemm<<<grid, 256, 0, s>>>(A, n, ld, j0, jb);
      note_launches(1);
    }
  }
  return 0;
}

// Solve with the dense LU for nrhs columns, one CTA per column, the column
// held in shared memory.  Blocked by kSB columns: warp 0 solves the kSB x kSB
// diagonal block with shuffles (each lane holding its row of the block,
// loaded up front), then all warps apply the solved block to the remaining
// rows as one small GEMV whose loads are all independent.  Two barriers per
// block instead of two per column, and no load waits behind a barrier.
constexpr int kSB = 32;
constexpr int kLST = 512;

// x_blk <- D^{-1} x_blk for the triangular diagonal block starting at j0
// (jb <= 32 rows, lane i owns row j0 + i).  lower: forward substitution,
// else backward.  M(i, c) reads the block entry of row i, column c (block
// coordinates); rd: null for a unit diagonal, else the reciprocals of the
// block's diagonal (multiplications in place of divisions).
template <class Get>
__device__ __forceinline__ void diag_block_solve(double *b, int j0, int jb,
                                                 bool lower,
                                                 const double *rd, Get M) {
  const int lane = threadIdx.x & 31;
  double row[kSB];
#pragma unroll
  for (int c = 0; c < kSB; ++c) row[c] = (lane < jb && c < jb) ? M(lane, c) : 0.0;
  double v = lane < jb ? b[j0 + lane] : 0.0;
  if (lower) {
#pragma unroll
    for (int c = 0; c < kSB; ++c) {
      if (c >= jb) break;
      if (rd && lane == c) v *= rd[c];
      const double xc = __shfl_sync(0xffffffffu, v, c);
      if (lane > c) v -= row[c] * xc;
    }
  } else {
#pragma unroll
    for (int c = kSB - 1; c >= 0; --c) {
      if (c >= jb) continue;
      if (rd && lane == c) v *= rd[c];
      const double xc = __shfl_sync(0xffffffffu, v, c);
      if (lane < c) v -= row[c] * xc;
    }
  }
  if (lane < jb) b[j0 + lane] = v;
}

__global__ void __launch_bounds__(kLST)
k_lu_solve(const double *LU, int n, int ld, const int32_t *piv, double *B,
           int ldb, int trans, const double *rdiag) {
  extern __shared__ double sb[];
  double *bg = B + (int64_t)ldb * blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int nw = kLST / 32;
  for (int i = tid; i < n; i += kLST) sb[i] = bg[i];
  __syncthreads();
  auto L = [&](int i, int j) { return LU[i + (int64_t)j * ld]; };
  if (!trans) {
    // P b, then L y = P b (unit lower), then U x = y
    if (tid == 0)
      for (int j = 0; j < n; ++j) {
        const int p = piv[j];
        if (p != j) {
          const double t = sb[j];
          sb[j] = sb[p];
          sb[p] = t;
        }
      }
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += kSB) {
      const int jb = min(kSB, n - j0);
      if (warp == 0)
        diag_block_solve(sb, j0, jb, true, nullptr,
                         [&](int i, int c) { return L(j0 + i, j0 + c); });
      __syncthreads();
      for (int i = j0 + jb + tid; i < n; i += kLST) {  // rows below
        // every load issued before the first product
        const double *li = LU + i + (int64_t)j0 * ld;
        double lv[kSB];
#pragma unroll
        for (int c = 0; c < kSB; ++c)
          lv[c] = c < jb ? __ldg(li + (int64_t)c * ld) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < kSB; ++c)
          acc += lv[c] * (c < jb ? sb[j0 + c] : 0.0);
        sb[i] -= acc;
      }
      __syncthreads();
    }
    for (int j0 = ((n - 1) / kSB) * kSB; j0 >= 0; j0 -= kSB) {
      const int jb = min(kSB, n - j0);
      if (warp == 0)
        diag_block_solve(sb, j0, jb, false, rdiag + j0,
                         [&](int i, int c) { return L(j0 + i, j0 + c); });
      __syncthreads();
      for (int i = tid; i < j0; i += kLST) {  // rows above
        const double *li = LU + i + (int64_t)j0 * ld;
        double lv[kSB];
#pragma unroll
        for (int c = 0; c < kSB; ++c)
          lv[c] = c < jb ? __ldg(li + (int64_t)c * ld) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < kSB; ++c)
          acc += lv[c] * (c < jb ? sb[j0 + c] : 0.0);
        sb[i] -= acc;
      }
      __syncthreads();
    }
  } else {
    // A^T = U^T L^T P: U^T z = b (lower, U's diagonal), L^T w = z (unit
    // upper), x = P^T w.  Rows of U^T / L^T are columns of LU: one warp per
    // row reads them coalesced.
    for (int j0 = 0; j0 < n; j0 += kSB) {
      const int jb = min(kSB, n - j0);
      if (warp == 0)
        diag_block_solve(sb, j0, jb, true, rdiag + j0,
                         [&](int i, int c) { return L(j0 + c, j0 + i); });
      __syncthreads();
      for (int i0 = j0 + jb + 4 * warp; i0 < n; i0 += 4 * nw) {
        double t[4];  // four rows per warp at a time
#pragma unroll
        for (int u = 0; u < 4; ++u)
          t[u] = (lane < jb && i0 + u < n)
                     ? L(j0 + lane, i0 + u) * sb[j0 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            t[u] += __shfl_xor_sync(0xffffffffu, t[u], o);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i0 + u < n) sb[i0 + u] -= t[u];
      }
      __syncthreads();
    }
    for (int j0 = ((n - 1) / kSB) * kSB; j0 >= 0; j0 -= kSB) {
      const int jb = min(kSB, n - j0);
      if (warp == 0)
        diag_block_solve(sb, j0, jb, false, nullptr,
                         [&](int i, int c) { return L(j0 + c, j0 + i); });
      __syncthreads();
      for (int i0 = 4 * warp; i0 < j0; i0 += 4 * nw) {
        double t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          t[u] = (lane < jb && i0 + u < j0)
                     ? L(j0 + lane, i0 + u) * sb[j0 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            t[u] += __shfl_xor_sync(0xffffffffu, t[u], o);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i0 + u < j0) sb[i0 + u] -= t[u];
      }
      __syncthreads();
    }
    if (tid == 0)
      for (int j = n - 1; j >= 0; --j) {
        const int p = piv[j];
        if (p != j) {
          const double t = sb[j];
          sb[j] = sb[p];
          sb[p] = t;
        }
      }
    __syncthreads();
  }
  for (int i = tid; i < n; i += kLST) bg[i] = sb[i];
}

// Many right-hand sides on a large top block: blocked triangular solves
// over all SMs instead of one CTA per column re-reading the whole LU (the
// 1M-node case: n = 6397, 32 columns, 415 ms).  Per 32-row block, one warp
// per column solves the diagonal block, then tiled FP64 GEMMs update the
// rows below (forward) or above (backward); the LU is read about once per
// sweep.  Modes: 0 = L (unit lower, forward), 1 = U (upper, backward),
// 2 = U^T (lower, forward), 3 = L^T (unit upper, backward).
namespace {
using wide::MV;
__device__ MV top_factor(const double *LU, int ld, int mode) {
  return mode < 2 ? wide::colmajor(const_cast<double *>(LU), ld)
                  : wide::transposed(const_cast<double *>(LU), ld);
}
}  // namespace

__global__ void k_top_swaps(const int32_t *piv, int n, double *B, int ldb,
                            int nrhs, int reverse) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  double *b = B + (int64_t)ldb * c;
  for (int t = 0; t < n; ++t) {
    const int j = reverse ? n - 1 - t : t, p = piv[j];
    if (p != j) {
      const double x = b[j];
      b[j] = b[p];
      b[p] = x;
    }
  }
}

__global__ void k_top_diag(const double *LU, int n, int ld, double *B,
                           int ldb, int nrhs, int j0, int mode,
                           const double *rdiag) {
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nrhs) return;  // whole warps
  const int jb = n - j0 < wide::kWNB ? n - j0 : wide::kWNB;
  const MV M = top_factor(LU, ld, mode);
  const MV Bv = wide::colmajor(B, ldb);
  const bool lower = mode == 0 || mode == 2, unit = mode == 0 || mode == 3;
  double x = lane < jb ? Bv.at(j0 + lane, c) : 0.0;
  if (lower) {
    for (int jj = 0; jj < jb; ++jj) {
      if (!unit && lane == jj) x *= rdiag[j0 + jj];
      const double xj = __shfl_sync(0xffffffffu, x, jj);
      if (lane > jj && lane < jb) x -= M.at(j0 + lane, j0 + jj) * xj;
    }
  } else {
    for (int jj = jb - 1; jj >= 0; --jj) {
      if (!unit && lane == jj) x *= rdiag[j0 + jj];
      const double xj = __shfl_sync(0xffffffffu, x, jj);
      if (lane < jj) x -= M.at(j0 + lane, j0 + jj) * xj;
    }
  }
  if (lane < jb) Bv.at(j0 + lane, c) = x;
}

__global__ void __launch_bounds__(256)
k_top_upd(const double *LU, int n, int ld, double *B, int ldb, int nrhs,
          int j0, int mode) {
  const int jb = n - j0 < wide::kWNB ? n - j0 : wide::kWNB;
  const bool lower = mode == 0 || mode == 2;
  const int lo = lower ? j0 + jb : 0, rows = lower ? n - lo : j0;
  const int r0 = blockIdx.x * wide::kWT, c0 = blockIdx.y * wide::kWT;
  if (r0 >= rows || c0 >= nrhs) return;
  const MV M = top_factor(LU, ld, mode);
  const MV Bv = wide::colmajor(B, ldb);
  const MV C = Bv.sub(lo, 0);
  wide::tile_gemm(C, C, M.sub(lo, j0), Bv.sub(j0, 0), rows, nrhs, jb, -1.0,
                  r0, c0);
}

static void top_trsm(const double *LU, int n, int ld, double *B, int ldb,
                     int nrhs, int mode, cudaStream_t s) {
  const bool lower = mode == 0 || mode == 2;
  const int nblk = (n + wide::kWNB - 1) / wide::kWNB;
  const unsigned gr = (unsigned)((n + wide::kWT - 1) / wide::kWT);
  const unsigned gc = (unsigned)((nrhs + wide::kWT - 1) / wide::kWT);
  for (int b = 0; b < nblk; ++b) {
    const int j0 = (lower ? b : nblk - 1 - b) * wide::kWNB;
    k_top_diag<<<(unsigned)((nrhs * 32 + 255) / 256), 256, 0, s>>>(
        LU, n, ld, B, ldb, nrhs, j0, mode, lu_rdiag(LU, n, ld));
    k_top_upd<<<dim3(gr, gc), 256, 0, s>>>(LU, n, ld, B, ldb, nrhs, j0,
                                           mode);
    note_launches(2);
  }
}

void launch_dense_lu_solve(const double *LU, int n, int ld, const int32_t *piv,
                           double *B, int ldb, int nrhs, int trans,
                           cudaStream_t s) {
  if (nrhs == 0 || n == 0) return;
  if (nrhs >= 4 && n >= 1024) {
    const unsigned gs = (unsigned)((nrhs + 127) / 128);
    if (!trans) {
      k_top_swaps<<<gs, 128, 0, s>>>(piv, n, B, ldb, nrhs, 0);
      note_launches(1);
      top_trsm(LU, n, ld, B, ldb, nrhs, 0, s);
      top_trsm(LU, n, ld, B, ldb, nrhs, 1, s);
    } else {
      top_trsm(LU, n, ld, B, ldb, nrhs, 2, s);
      top_trsm(LU, n, ld, B, ldb, nrhs, 3, s);
      k_top_swaps<<<gs, 128, 0, s>>>(piv, n, B, ldb, nrhs, 1);
      note_launches(1);
    }
    return;
  }
  const size_t sm = (size_t)n * 8;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_lu_solve,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_lu_solve<<<nrhs, kLST, sm, s>>>(LU, n, ld, piv, B, ldb, trans,
                                    lu_rdiag(LU, n, ld));
  note_launches(1);
}

// ---------------------------------------------------------------------------
// top-level right-hand side and back substitution (Eq. partition)

// partial[chunk][q][a] = sum over the chunk's rows r with rmask[r] of
// C[r, a] b[r, q]: CTA (row chunk, 32 columns a, up to kTQ columns q).
// Per slab of kTS rows the C tile and the b rows are staged in shared
// memory with loads along the rows (coalesced); a slab whose masked C tile
// is zero (the Psi-derived columns are zero away from their hole's boxes)
// skips its b loads and products.  Thread (a = lane, warp g) sums rows
// g*8 .. g*8+7 of each slab; the 8 warp sums are added in a fixed order.
__global__ void __launch_bounds__(256)
k_top_rhs_part(const double *b, int64_t ldb, int nrhs, const double *C,
               int64_t ldc, int p3, const uint8_t *rmask, int64_t n2,
               int64_t rows, double *partial) {
  __shared__ double Cs[32][kTS + 1];
  __shared__ double Bs[kTQ][kTS + 1];
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  const int a0 = blockIdx.y * 32, q0 = blockIdx.z * kTQ;
  const int nq = nrhs - q0 < kTQ ? nrhs - q0 : kTQ;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = r0 + rows < n2 ? r0 + rows : n2;
  double acc[kTQ];
#pragma unroll
  for (int q = 0; q < kTQ; ++q) acc[q] = 0.0;
  for (int64_t s0 = r0; s0 < r1; s0 += kTS) {
    bool nz = false;
#pragma unroll
    for (int u = 0; u < 32 * kTS / 256; ++u) {
      const int idx = tid + 256 * u, r = idx % kTS, a = idx / kTS;
      const int64_t row = s0 + r;
      double v = 0.0;
      if (row < r1 && a0 + a < p3 && rmask[row]) v = C[row + ldc * (a0 + a)];
      Cs[a][r] = v;
      nz |= v != 0.0;
    }
    if (!__syncthreads_or(nz)) continue;
    for (int idx = tid; idx < kTQ * kTS; idx += 256) {
      const int r = idx % kTS, q = idx / kTS;
      const int64_t row = s0 + r;
      Bs[q][r] = (row < r1 && q < nq) ? b[row + ldb * (q0 + q)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kTS / 8; ++j) {
      const int r = g * (kTS / 8) + j;
      const double c = Cs[lane][r];
#pragma unroll
      for (int q = 0; q < kTQ; ++q)
        if (q < nq) acc[q] += c * Bs[q][r];
    }
    __syncthreads();
  }
  // fixed-order sum of the 8 warps, 8 right-hand sides at a time
  double *red = &Cs[0][0];  // 8 x 32 x 8 doubles
  const int64_t base = (int64_t)blockIdx.x * nrhs;
#pragma unroll
  for (int qc = 0; qc < kTQ; qc += 8) {
    if (qc < nq) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 8; ++j) red[(g * 32 + lane) * 8 + j] = acc[qc + j];
      __syncthreads();
      const int q = qc + g;
      if (q < nq && a0 + lane < p3) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[(w * 32 + lane) * 8 + g];
        partial[(base + q0 + q) * p3 + a0 + lane] = v;
      }
    }
  }
}

// rhs[0:s] = b[root_act]; rhs[s + a] = g[a] - sum over chunks of the
// partials, one warp per (a, q) summing the chunks lane-strided and then a
// fixed shuffle tree.
__global__ void k_top_rhs_final(const double *b, int64_t ldb, int nrhs,
                                const int32_t *root_act, int s, int p3,
                                int nchunk, const double *partial,
                                const double *gsrc, int64_t ldg, double *rhs,
                                int ldr) {
  const int q = blockIdx.y;
  const int spad = (s + 31) & ~31;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < spad) {
    if (t < s) rhs[t + (int64_t)ldr * q] = b[root_act[t] + ldb * q];
    return;
  }
  const int64_t u = t - spad;
  const int a = (int)(u >> 5), lane = (int)(u & 31);
  if (a >= p3) return;  // whole warps
  double v = 0.0;
  for (int c = lane; c < nchunk; c += 32)
    v += partial[((int64_t)c * nrhs + q) * p3 + a];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) rhs[s + a + (int64_t)ldr * q] = gsrc[a + ldg * q] - v;
}

void launch_top_rhs(const double *b, int64_t ldb, int nrhs,
                    const int32_t *root_act, int s, const double *C,
                    int64_t ldc, int p3, const uint8_t *rmask, int64_t n2,
                    const double *gsrc, int64_t ldg, double *partial,
                    double *rhs, int ldr, cudaStream_t st) {
  if (nrhs == 0) return;
  const int nchunk = top_rhs_chunks(n2, p3, nrhs);
  if (p3 > 0 && n2 > 0) {
    const dim3 grid((unsigned)nchunk, (unsigned)((p3 + 31) / 32),
                    (unsigned)((nrhs + kTQ - 1) / kTQ));
    k_top_rhs_part<<<grid, 256, 0, st>>>(b, ldb, nrhs, C, ldc, p3, rmask, n2,
                                         top_rhs_rows(n2, p3, nrhs), partial);
    note_launches(1);
  } else if (p3 > 0) {
    cudaMemsetAsync(partial, 0, sizeof(double) * nrhs * p3, st);
  }
  const int64_t tot = ((s + 31) & ~31) + 32 * (int64_t)p3;
  k_top_rhs_final<<<dim3((unsigned)((tot + 255) / 256), nrhs), 256, 0, st>>>(
      b, ldb, nrhs, root_act, s, p3, n2 > 0 ? nchunk : 1, partial, gsrc, ldg,
      rhs, ldr);
  note_launches(1);
}

// y[r, q] -= sum_a W[r, a] lambda[a, q] for the rows with rmask set, lambda
// = top[s:s+p3, q]: one thread per row (the W loads run along the rows,
// coalesced), up to kTQ right-hand sides per CTA held in registers, lambda
// staged 32 border columns at a time in shared memory (broadcast reads).
// A warp skips the products of a column that is zero on all its rows (the
// Psi-derived columns of the adjoint).  The same launch writes the rows
// that are not swept: y[root_act[i]] = top[i] and y[n2 + a] = lambda[a].
__global__ void __launch_bounds__(256)
k_top_back(double *y, int64_t ldy, int nrhs, const int32_t *root_act, int s,
           const double *W, int64_t ldw, int p3, const uint8_t *rmask,
           int64_t n2, const double *top, int ldt) {
  __shared__ double Ls[32][kTQ + 1];
  const int tid = threadIdx.x;
  const int q0 = blockIdx.y * kTQ;
  const int nq = nrhs - q0 < kTQ ? nrhs - q0 : kTQ;
  const int64_t i = (int64_t)blockIdx.x * 256 + tid;
  for (int q = 0; q < nq; ++q) {  // rows outside the sweep
    const double *col = top + (int64_t)ldt * (q0 + q);
    if (i < s) y[root_act[i] + ldy * (q0 + q)] = col[i];
    else if (i < s + p3) y[n2 + (i - s) + ldy * (q0 + q)] = col[i];
  }
  if ((int64_t)blockIdx.x * 256 >= n2) return;  // whole CTAs
  const int64_t row = i;
  const bool live = row < n2 && rmask[row];
  double acc[kTQ];
#pragma unroll
  for (int q = 0; q < kTQ; ++q) acc[q] = 0.0;
  for (int a0 = 0; a0 < p3; a0 += 32) {
    __syncthreads();
    for (int idx = tid; idx < 32 * kTQ; idx += 256) {
      const int a = idx % 32, q = idx / 32;
      Ls[a][q] = (a0 + a < p3 && q < nq)
                     ? top[s + a0 + a + (int64_t)ldt * (q0 + q)]
                     : 0.0;
    }
    __syncthreads();
    const int na = p3 - a0 < 32 ? p3 - a0 : 32;
#pragma unroll 2
    for (int a = 0; a < na; ++a) {
      const double w = live ? W[row + ldw * (a0 + a)] : 0.0;
      if (__any_sync(0xffffffffu, w != 0.0)) {
#pragma unroll
        for (int q = 0; q < kTQ; ++q)
          if (q < nq) acc[q] += w * Ls[a][q];
      }
    }
  }
  if (live)
#pragma unroll
    for (int q = 0; q < kTQ; ++q)
      if (q < nq) y[row + ldy * (q0 + q)] -= acc[q];
}

void launch_top_back(double *y, int64_t ldy, int nrhs, const int32_t *root_act,
                     int s, const double *W, int64_t ldw, int p3,
                     const uint8_t *rmask, int64_t n2, const double *top,
                     int ldt, cudaStream_t st) {
  if (nrhs == 0) return;
  int64_t bx = (n2 + 255) / 256;
  const int64_t bp = (s + p3 + 255) / 256;
  if (bp > bx) bx = bp;
  k_top_back<<<dim3((unsigned)bx, (unsigned)((nrhs + kTQ - 1) / kTQ)), 256,
               0, st>>>(y, ldy, nrhs, root_act, s, W, ldw, p3, rmask, n2, top,
                        ldt);
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
