// Internal declarations shared by the host runtime (C++) and the CUDA
// kernels of the skeletonization solver.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "skel.h"

namespace skel {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// geometry on the device (structure of arrays, caller's node order)
struct DevGeom {
  int64_t N;
  int32_t p;
  // kernel family: 0 = Stokes double layer (2 DOFs per node, bordered),
  // 1 = Laplace Neumann single-layer form (1 DOF per node, no bordering)
  int32_t lap;
  const double *x, *y, *nx, *ny, *w, *kap;  // kap = (gamma''.n)/|gamma'|^2
  const int32_t *comp;
  const double *centers;                      // p x 2
  // FP32 copies for the mixed-precision form: positions as float pairs
  // x = xh + xl (exact to ~2^-48 relative), the rest rounded to float
  const float *xh, *xl, *yh, *yl, *nxf, *nyf, *wf, *kapf;
};

// Persistent per-box factor record (indexed by box id, all levels).
//   dofs[dof_off .. dof_off+n): active DOFs, skeleton first then redundant
//   fac[fac_off ..): T (k x r, ld k) | Y (r x k, ld r) | Z (k x r, ld k) |
//                    LU(X_RR) (r x r, ld r) | X_SS (k x k, ld k)
//   ipool[piv_off .. +r): LU row interchanges (LAPACK style, 0-based)
struct DevBox {
  int32_t n, k;
  int64_t dof_off, fac_off, piv_off;
  int32_t leaf;      // a leaf box (its sweep inputs come from the data)
  int32_t pad;
  int64_t snap_off;  // bordered-sweep snapshot region (2 k x 3p doubles)
};

__host__ __device__ inline int64_t fac_T(int k, int r) { return 0; }
__host__ __device__ inline int64_t fac_Y(int k, int r) { return (int64_t)k * r; }
__host__ __device__ inline int64_t fac_Z(int k, int r) { return 2 * (int64_t)k * r; }
__host__ __device__ inline int64_t fac_LU(int k, int r) { return 3 * (int64_t)k * r; }
__host__ __device__ inline int64_t fac_XSS(int k, int r) {
  return 3 * (int64_t)k * r + (int64_t)r * r;
}
// upper bound of the region: n^2 + k r <= 1.25 n^2
__host__ __device__ inline int64_t fac_region(int n) {
  return (int64_t)n * n + ((int64_t)n * n + 3) / 4 + 8;
}

// One box of the level being compressed.
struct LvlBox {
  int32_t box;               // box id
  int32_t n, m, nf;          // active DOFs, ID-matrix rows, near-field DOFs
  int32_t nchild;
  int32_t cseg[4];           // child segment start in the active list
  int32_t ck[4];             // child skeleton size
  int64_t cxss[4];           // child X_SS offset in fac
  int64_t act_off, fint_off; // into the level's int scratch
  int64_t a_off, m_off;      // into the level's double scratch
  int64_t perm_off;          // into the level's int scratch (CPQR permutation)
  int64_t t_off;             // FP64 workspace for T (k x r <= n^2/4 doubles)
  double cx, cy, rho;        // proxy circle
};

// ---------------------------------------------------------------------------
// host quadtree (Sec. 2.3)
struct HBox {
  int depth;
  int64_t ix, iy;
  double cx, cy, hw;
  int parent;
  int child[4];
  int nchild;
  int64_t nbeg, ncnt;        // subtree nodes: Tree::order[nbeg .. nbeg+ncnt)
  bool leaf;
};

struct Tree {
  std::vector<HBox> boxes;
  std::vector<std::vector<int>> levels;
  std::vector<int64_t> order;   // node ids, each box's subtree contiguous,
                                // ascending ids inside every box
  std::unordered_map<uint64_t, int> key2id;
  int L() const { return (int)levels.size() - 1; }
};

inline uint64_t box_key(int depth, int64_t ix, int64_t iy) {
  return ((uint64_t)depth << 58) ^ ((uint64_t)ix << 29) ^ (uint64_t)iy;
}

// Build the tree from host positions.  Root: bounding square of Gamma_0
// (comp == 0) with a 1% margin.  Returns false (and sets err) when a node
// lies outside the root box or no node belongs to Gamma_0.
bool build_tree(const double *x, const double *y, const int32_t *comp,
                int64_t N, int leaf_size, Tree &t, std::string &err);

// Same as build_tree but with an explicit root square.
void build_tree_root(const double *x, const double *y, int64_t N,
                     int leaf_size, double cx, double cy, double hw, Tree &t);

// Owners of active DOFs at the start of `level` (boxes of that depth and
// leaves above it) other than b whose square meets b's proxy disk.
void near_owners(const Tree &t, int b, int level, double ratio,
                 std::vector<int> &out);

inline double proxy_radius(const HBox &B, double ratio) {
  return ratio * 1.4142135623730951 * B.hw;
}

// ---------------------------------------------------------------------------
// device memory through the process-wide cache of freed blocks (pool.cpp)
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
double dev_alloc_ms();     // host time spent in dev_alloc / dev_free so far
size_t dev_cached_bytes();

// ---------------------------------------------------------------------------
// kernel launchers (CUDA translation units).  Every launcher reports the
// kernels it starts through note_launches (process-wide counter).
void note_launches(int n);
// f32 receives 8 arrays of N floats: xh, xl, yh, yl, nx, ny, w, kap
void launch_quadrature(const double *x, const double *y, const double *dx,
                       const double *dy, const double *ddx, const double *ddy,
                       const double *dt, int64_t N, double *nx, double *ny,
                       double *w, double *kap, float *f32, cudaStream_t s);

// Box compression for the FP64 form (Real = double) and the mixed form
// (Real = float); the factor and scratch pools are addressed in Real units.
template <class Real>
void launch_assemble_diag(const DevGeom &g, const LvlBox *lb, int nbox,
                          const int32_t *iscr, Real *dscr, const Real *fac,
                          cudaStream_t s);
template <class Real>
void launch_assemble_id(const DevGeom &g, const LvlBox *lb, int nbox,
                        const int32_t *iscr, Real *dscr, int n_proxy,
                        cudaStream_t s);
// one CTA per box: sel[0..nbox) indexes lb; tws is the FP64 T workspace
// (ID matrix stored as Real, T stored as Fac)
template <class Real, class Fac>
void launch_cpqr(const LvlBox *lb, const int32_t *sel, int nbox,
                 int32_t *iscr, Real *dscr, DevBox *boxes, Fac *fac,
                 double *tws, double tol, int max_n, cudaStream_t s);
// X_RR conditioning (Sec. 2.2 remark): an LU pivot of X_RR at or below
// kMoveRatio of the largest flags the box (flag[q] = 1, elimination stops
// after the LU when allow_move != 0); launch_xrr_split_cluster then finds
// the indices to move from R into S (moves[q] of them, ascending in the
// box's pivot slot) and launch_repartition applies the move.
constexpr double kMoveRatio = 1e-3;
template <class Real>
void launch_eliminate(const LvlBox *lb, const int32_t *sel, int nbox,
                      const int32_t *iscr, const Real *dscr, DevBox *boxes,
                      Real *fac, int32_t *ipool, int32_t *dofs, int max_n,
                      int *status, int allow_move, int32_t *flag,
                      cudaStream_t s);
template <class Fac>
void launch_repartition(const LvlBox *lb, const int32_t *sel, int nbox,
                        int32_t *iscr, DevBox *boxes, Fac *fac,
                        const int32_t *ipool, const int32_t *moves,
                        double *tws, int64_t tws_half, int max_n,
                        cudaStream_t s);
// one thread-block cluster per box: cs = 16 CTAs for large boxes, 4 for
// mid-size ones (the X_RR split always uses 16)
int cluster_size();
template <class Real, class Fac>
cudaError_t launch_cpqr_cluster(const LvlBox *lb, const int32_t *sel, int nsel,
                                int32_t *iscr, Real *dscr, DevBox *boxes,
                                Fac *fac, double *tws, double tol, int max_n,
                                int max_m, cudaStream_t s, int cs);
template <class Real>
cudaError_t launch_eliminate_cluster(const LvlBox *lb, const int32_t *sel,
                                     int nsel, const int32_t *iscr,
                                     const Real *dscr, DevBox *boxes,
                                     Real *fac, int32_t *ipool, int32_t *dofs,
                                     int max_n, int *status, int allow_move,
                                     int32_t *flag, cudaStream_t s, int cs);
template <class Real>
cudaError_t launch_xrr_split_cluster(const LvlBox *lb, const int32_t *sel,
                                     int nsel, const int32_t *iscr,
                                     const Real *dscr, DevBox *boxes,
                                     Real *fac, int32_t *ipool,
                                     int32_t *moves, int max_n,
                                     cudaStream_t s);
// 3xTF32 tensor-core GEMM (k_tc.cu): C = C0 + sign A B for strided FP64
// views (element (i, j) of a view at p[i rs + j cs]); the job lives in
// device memory so that its sizes may be set by an earlier kernel.  The
// grid covers max_m x max_n; a timed-out wait sets *err = SKEL_ETIMEOUT.
struct TcView {
  const double *p;
  int64_t rs, cs;
};
struct TcJob {
  TcView A, B, C0;
  double *C;
  int64_t c_rs, c_cs;
  int M, N, K;
  double sign;
};
cudaError_t launch_tc_gemm(const TcJob *job, int max_m, int max_n, int *err,
                           cudaStream_t s);
// Elimination of large boxes (FP64 factors) by whole-GPU launches, one box
// after another on stream s (k_wide.cu): qs are positions in lb, ns their
// active DOF counts; Kp holds max(ns)^2 doubles, ops qs.size() descriptors
// of wide_ops_bytes() each.  Same results layout, flags and status as
// launch_eliminate.
struct WideOps;
size_t wide_ops_bytes();
// Box b runs on streams[b % streams.size()] with its own gathered block
// in Kp (streams.size() x max(ns)^2 doubles).  With allow_move the boxes'
// X_RR is kept in Xs (qs.size() x max(ns)^2 doubles) for
// launch_xrr_split_wide; iws holds 2 max(ns) ints per box.
cudaError_t launch_eliminate_wide(const LvlBox *lb, const std::vector<int> &qs,
                                  const std::vector<int> &ns,
                                  const int32_t *iscr, const double *dsa,
                                  DevBox *boxes, double *fac, int32_t *ipool,
                                  int32_t *dofs, double *Kp, double *Xs,
                                  int32_t *iws, WideOps *ops, int *status,
                                  int allow_move, int32_t *flag, bool tc,
                                  const std::vector<cudaStream_t> &streams);
// Column-pivoted QR (ID) of wide boxes with whole-GPU launches
// (k_wide_qr.cu): results as launch_cpqr_cluster.  qs, ns, ms: positions
// in lb, active DOFs and ID-matrix rows; box b on streams[b % size];
// ops: qs.size() descriptors of qr_ops_bytes(); dws: 2 max(ns) doubles and
// iws: max(ns) ints per box; R: streams.size() x max(ns)^2 doubles;
// hstop: 2 qs.size() pinned ints and events 2 qs.size() events for the
// host's reads of the stop flags.
struct QrOps;
size_t qr_ops_bytes();
template <class Real, class Fac>
cudaError_t launch_cpqr_wide(const LvlBox *lb, const std::vector<int> &qs,
                             const std::vector<int> &ns,
                             const std::vector<int> &ms, int32_t *iscr,
                             Real *dscr, DevBox *boxes, Fac *fac,
                             double *tws, double tol, QrOps *ops,
                             double *dws, int32_t *iws, double *R,
                             const std::vector<cudaStream_t> &streams,
                             volatile int32_t *hstop,
                             const std::vector<cudaEvent_t> &events);
// the X_RR split (as launch_xrr_split_cluster) of flagged wide boxes: qs
// and ns as in the elimination pass that flagged them, bidx[b] the box's
// position in that pass (its descriptor ops[bidx[b]]); box b runs on
// streams[b % streams.size()], the boxes' steps enqueued in turn
cudaError_t launch_xrr_split_wide(const LvlBox *lb,
                                  const std::vector<int> &qs,
                                  const std::vector<int> &ns,
                                  const std::vector<int> &bidx,
                                  const DevBox *boxes, int32_t *ipool,
                                  WideOps *ops, int32_t *moves,
                                  const std::vector<cudaStream_t> &streams);
// the root block (FP64) from children's Schur complements stored as Real
template <class Real>
void launch_root_block(const DevGeom &g, const LvlBox *lb, const int32_t *iscr,
                       const Real *fac, double *top, int ld, cudaStream_t s);
void launch_h_columns(const DevGeom &g, double *H, int64_t ld, cudaStream_t s);
void launch_psi_columns(const DevGeom &g, double *P, int64_t ld,
                        cudaStream_t s);
void launch_point_force_rhs(const DevGeom &g, int nrhs, int ns,
                            const double *sxy, const double *sf,
                            int holes_zero, double *f, int64_t ld,
                            cudaStream_t s);
// FP64 vector kernels of the refinement loop (k_blas.cu)
size_t multidot_scratch();
// out[c] = x . Y[:, c] for c < ncol <= 64 (out on the device)
void launch_multidot(const double *x, const double *Y, int64_t ld, int ncol,
                     int64_t n, double *part, double *out, cudaStream_t s);
// y <- a y + csign * sum_c coef[c] X[:, c]
void launch_combine(double *y, double a, const double *X, int64_t ld,
                    const double *coef, double csign, int ncol, int64_t n,
                    cudaStream_t s);
void launch_axpby(double alpha, const double *x, double beta, double *y,
                  int64_t n, cudaStream_t s);

// Double-layer sums are split over source chunks; the partial sums need
// dl_scratch(nt, nrhs, N) doubles of scratch.
size_t dl_scratch(int64_t nt, int nrhs, int64_t N);
// source chunks for a pair-sum grid of units x chunks CTAs, chosen so that
// the CTAs spread evenly over the SMs (k_geom.cu)
int balanced_chunks(int64_t units, int64_t maxc, int min_per_sm);
void launch_eval_velocity(const DevGeom &g, int nrhs, const double *sol,
                          int64_t ld, int64_t nt, const double *tx,
                          const double *ty, double *u, double *scratch,
                          cudaStream_t s);
bool launch_eval_velocity_capped(const DevGeom &g, int nrhs, const double *sol,
                                 int64_t ld, int64_t nt, const double *tx,
                                 const double *ty, double *u, double *scratch,
                                 int64_t cap, cudaStream_t s);
// skel_eval_velocity_noalloc (k_noalloc.cu): the velocity sums with their
// partial sums in a fixed device array of kNoallocScratchDoubles, whose
// address is resolved once per device on first use.
constexpr int64_t kNoallocScratchDoubles = 524288;  // 4 MiB
int launch_eval_velocity_noalloc(const DevGeom &g, int nrhs, const double *sol,
                                 int64_t ld, int64_t nt, const double *tx,
                                 const double *ty, double *u, cudaStream_t s,
                                 std::string &err);
// Laplace Neumann form: y = (1/2 I + D + N) x (scratch: nrhs doubles) and
// u = S sol at nt targets (u: nt x nrhs, ld nt)
void launch_lap_matvec(const DevGeom &g, int nrhs, const double *x, double *y,
                       int64_t ld, double *scratch, cudaStream_t s);
void launch_lap_potential(const DevGeom &g, int nrhs, const double *sol,
                          int64_t ld, int64_t nt, const double *tx,
                          const double *ty, double *u, cudaStream_t s);
void launch_matvec(const DevGeom &g, int nrhs, const double *x, double *y,
                   int64_t ld, double *scratch, cudaStream_t s);
// Operator apply with the O(N^2) double-layer sums in double-float
// arithmetic (k_dlf.cu), one column.  blk: nblk pairs (first node, count)
// covering the nodes, each at most dlf_block_size() nodes of one curve;
// scratch: dlf_scratch(N, nblk) doubles.
int dlf_block_size();
size_t dlf_scratch(int64_t N, int nblk);
// the double-float pair sums into partial slots; returns the slot count
int launch_dlf_sym(const DevGeom &g, const double *mu, const int32_t *blk,
                   int nblk, double *partial, cudaStream_t s);
// the transposed sums (partials carry w_t / pi); returns the slot count
int launch_dlfT_sym(const DevGeom &g, const double *z, const int32_t *blk,
                    int nblk, double *partial, cudaStream_t s);
// A^T z (one column) with the transposed sums in double-float arithmetic
void launch_matvec_fast_adjoint(const DevGeom &g, const double *z, double *y,
                                const int32_t *blk, int nblk, double *scratch,
                                cudaStream_t s);
void launch_matvec_fast(const DevGeom &g, const double *x, double *y,
                        const int32_t *blk, int nblk, double *scratch,
                        cudaStream_t s);
void launch_matvec_adjoint(const DevGeom &g, int nrhs, const double *z,
                           double *y, int64_t ld, double *scratch,
                           cudaStream_t s);

// Shape derivatives (k_grad.cu): L = z^T A s and ubar . E s with respect
// to the samples (6N: x, y, gamma', gamma'') and the centres (2p) written
// to out (6N + 2p); the velocity form also writes gs = E^T ubar.  Scratch:
// grad_scratch(N, nt) doubles.
size_t grad_scratch(int64_t N, int64_t nt);
// ranges of the symmetric pair sums over the nodes: R ranges of S points
// (S a multiple of 128, about 64 ranges)
void sym_ranges(int64_t N, int &S, int &R);
void launch_grad_bilinear(const DevGeom &g, const double *dx, const double *dy,
                          const double *ddx, const double *ddy,
                          const double *dt, const double *z, const double *s,
                          double *scratch, double *out, cudaStream_t st);
void launch_grad_velocity(const DevGeom &g, const double *dx,
                          const double *dy, const double *dt, const double *s,
                          int64_t nt, const double *tx, const double *ty,
                          const double *ubar, double *scratch, double *gs,
                          double *out, cudaStream_t st);

// sweeps over one level's boxes (box ids in `ids`)
//   mode 0: U   (b_R -= T^T b_S; b_S -= Z b_R; b_R <- X_RR^{-1} b_R)
//   mode 1: V^T (b_R -= T^T b_S; b_S -= Y^T b_R; b_R <- X_RR^{-T} b_R)
// `pre` (may be null) receives b_R before the X_RR solve.
// Factors are stored as Real; vectors are always FP64.  qmax caps the
// right-hand sides per CTA (4, 8 or 16; a tuning parameter).  One launch sweeps
// up to two independent jobs (right-hand-side sets of nrhs columns with
// leading dimension ld, each with its own mode) over the same factors.
struct UpJobs {
  double *b[2];
  double *pre[2];
  int mode[2];
  // bordered sweeps only (nullptr otherwise): the initial columns read by
  // leaf boxes instead of b, and the snapshot arena receiving every swept
  // box's b_S output (region snap_off + job * k * nrhs, column-major k rows)
  const double *init[2];
  double *snap;
};
// Work items of a bordered sweep: (box id, right-hand-side chunk, job)
// triples; the chunk width is sweep_chunk() of the whole level, so a box
// swept alone gives the same bits as in a sweep of its level.
int sweep_chunk(int nbox, int njobs, int nrhs, int max_n, int qmax);
// Acc: the sweep's arithmetic (double, or float for the mixed form's
// bordered sweeps); the vectors in global memory are FP64 either way
template <class Real, class Acc>
void launch_up_items(const DevBox *boxes, const int32_t *items, int nitems,
                     const int32_t *dofs, const Real *fac,
                     const int32_t *ipool, const UpJobs &jobs, int64_t ld,
                     int nrhs, int q, int max_n, int *status, cudaStream_t s);
// b_S rows of skipped boxes put back into the sweep columns from their
// snapshots, for the parents that are swept again (items as above)
void launch_snap_restore(const DevBox *boxes, const int32_t *items, int nitems,
                         const int32_t *dofs, const UpJobs &jobs, int64_t ld,
                         int nrhs, int q, cudaStream_t s);
template <class Real>
void launch_up_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                     const int32_t *dofs, const Real *fac,
                     const int32_t *ipool, const UpJobs &jobs, int njobs,
                     int64_t ld, int nrhs, int max_n, int qmax, int *status,
                     cudaStream_t s);
//   mode 0: V   (x_R -= Y x_S; x_S -= T x_R)
//   mode 1: U^T (x_R -= Z^T x_S; x_S -= T x_R)
template <class Real>
void launch_down_sweep(const DevBox *boxes, const int32_t *ids, int nbox,
                       const int32_t *dofs, const Real *fac, double *x,
                       int64_t ld, int nrhs, int mode, int max_n, int qmax,
                       int *status, cudaStream_t s);

// bordered top block
// row chunks of launch_top_rhs's partial products (nchunk x nrhs x p3
// doubles of scratch) for n2 swept rows
int top_rhs_chunks(int64_t n2, int p3, int nrhs);
// out (cols x cols) = A_R^T B_R over the rows with rmask set, skipping the
// zero rows of A's columns; scratch: gram_scratch_ints(rows, cols) ints
size_t gram_scratch_ints(int64_t rows, int cols);
void launch_gram_masked(const double *A, const double *B, int64_t rows,
                        int64_t ld, int cols, const uint8_t *rmask,
                        int32_t *scratch, double *out, cudaStream_t s);
void launch_top_fill(double *top, int ld, int s, int p3, const int32_t *root_act,
                     const double *UH, const double *QT, int64_t ldh,
                     const double *G, cudaStream_t s0);
// doubles the dense LU needs after A[ld * n] besides its 2 pivot statistics
int lu_map_doubles();
// doubles a dense LU of order n needs after A[ld * n]: its 2 pivot
// statistics, the panel row map and the reciprocals of U's diagonal
int lu_extra_doubles(int n);
int launch_dense_lu(double *A, int n, int ld, int32_t *piv, int *status,
                    cudaStream_t s);
void launch_dense_lu_solve(const double *LU, int n, int ld, const int32_t *piv,
                           double *B, int ldb, int nrhs, int trans,
                           cudaStream_t s);
// top-level right-hand side: rhs[0:s] = b[root_act]; rhs[s:] = g - C_R^T b_R
void launch_top_rhs(const double *b, int64_t ldb, int nrhs,
                    const int32_t *root_act, int s, const double *C,
                    int64_t ldc, int p3, const uint8_t *rmask, int64_t n2,
                    const double *gsrc, int64_t ldg, double *partial,
                    double *rhs, int ldr, cudaStream_t st);
// y_R -= W_R lambda; y[root_act] = top[0:s]; write lambda
void launch_top_back(double *y, int64_t ldy, int nrhs, const int32_t *root_act,
                     int s, const double *W, int64_t ldw, int p3,
                     const uint8_t *rmask, int64_t n2, const double *top,
                     int ldt, cudaStream_t st);
void launch_copy_cols(const double *src, int64_t lds, double *dst,
                      int64_t ldd, int64_t rows, int nrhs, cudaStream_t s);

}  // namespace skel
