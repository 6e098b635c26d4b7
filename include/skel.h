/*
 * skel.h -- C ABI of the GB300 recursive-skeletonization solver for the
 * 2-D Stokes double-layer equation on multiply-connected boundaries
 * (Ryan & Damle, "Parallel skeletonization for integral equations in
 * evolving multiply-connected domains").
 *
 * The solved system is the bordered Nystrom system of Sec. 3.1, Eq.
 * (backwardeq):
 *
 *     [ -1/2 I + D + N   H ] [ mu     ]   [ f ]
 *     [      Psi^T      -I ] [ lambda ] = [ g ]
 *
 * of size 2N + 3p (N boundary nodes, p holes).  D is the stresslet
 * double layer of Eq. (stokesbie) discretised by the trapezoid rule, N the
 * rank-one completion of Eq. (null-spaceop), H = [S R] the Stokeslet and
 * rotlet columns at the hole centres c_i, Psi the per-hole rigid motions of
 * Eq. (null-space), whose transpose acts as an integral.
 *
 * Conventions shared by every call
 *  - Status: 0 is success; negative values are the SKEL_E* codes below and
 *    skel_last_error() holds a one-line message.  No call aborts the process.
 *  - Pointers: every array argument may be host memory or CUDA device memory
 *    of the current device (the library copies with cudaMemcpyDefault).
 *    The caller owns every array it passes in and every output array; the
 *    context owns the tree and the factors, and frees them in skel_destroy.
 *  - Work is stream-ordered on the stream given to skel_build_tree; calls
 *    return after their results are in the output arrays.  skel_factor
 *    and the update calls run on an internal stream of the highest
 *    priority that waits for that stream on entry and that it waits for
 *    on return.
 *  - DOF order: node j's density is (mu_x, mu_y) at positions 2j, 2j+1 in
 *    the caller's node order; then lambda, hole-major
 *    (alpha_i1, alpha_i2, beta_i) for i = 1..p.
 *  - Matrices of right-hand sides are column-major with leading dimension
 *    2N + 3p.  A call takes at most 65535 columns (nrhs); more give
 *    SKEL_EINVAL.
 *  - All arithmetic is IEEE double on the GPU in the SKEL_FP64 form; the
 *    SKEL_MIXED form is described at skel_params.precision.
 */
#ifndef SKEL_H
#define SKEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SKEL_OK = 0,
  SKEL_EINVAL = -1,     /* bad argument (size, pointer, geometry)          */
  SKEL_ENOMEM = -2,     /* device allocation failed                         */
  SKEL_ECAPACITY = -3,  /* a box exceeded the kernels' size limits          */
  SKEL_ESINGULAR = -4,  /* a pivot of X_RR or of the top block vanished     */
  SKEL_ENOCONV = -5,    /* refinement did not reach its tolerance           */
  SKEL_ETIMEOUT = -6,   /* a bounded device wait gave up                    */
  SKEL_ECUDA = -7,      /* a CUDA runtime call failed                       */
  SKEL_ESTATE = -8      /* call out of order (e.g. solve before factor)     */
};

enum { SKEL_FP64 = 0, SKEL_MIXED = 1 };
/* Kernel families (skel_params.kernel). */
enum { SKEL_KERNEL_STOKES = 0, SKEL_KERNEL_LAPLACE = 1 };

typedef struct skel_ctx skel_ctx;

/* Factorization parameters.
 *  leaf_size   : maximum nodes per leaf box of the adaptive quadtree
 *                (Sec. 2.3).  Default 64.
 *  n_proxy     : points on each box's proxy circle (Sec. 2.5), 4..256.
 *                Default 64.
 *  proxy_ratio : proxy circle radius / box half-diagonal.  Default 1.5.
 *  id_tol      : interpolative-decomposition tolerance, relative to the
 *                first pivot of the column-pivoted QR (Sec. 2.2).
 *  precision   : SKEL_FP64: every step in IEEE double.
 *                SKEL_MIXED: the ID matrices and their Householder
 *                updates are computed and stored in FP32 (kernel entries
 *                from float-pair coordinate differences), while the
 *                column-norm bookkeeping, pivot choice and stopping test of
 *                the CPQR, the triangular solves forming T, the
 *                elimination and the bordered top block stay FP64 (the
 *                bordered sweeps run in FP32 arithmetic over them).  Solves
 *                then run GMRES on the FP64 operator preconditioned by
 *                these factors (the paper notes a looser factorization
 *                makes a good preconditioner, Eq. kinv remark).  An id_tol
 *                of 1e-6 .. 3e-7 suits FP32 IDs.  The environment variable
 *                SKEL_MIXED_FACTORS=fp32, read by skel_build_tree, also
 *                eliminates and stores the factors in FP32 (experimental:
 *                large top-level boxes can spoil the preconditioner).
 *  gmres_tol, gmres_maxit : SKEL_MIXED refinement: stop when the relative
 *                residual ||f - A x|| / ||f|| <= gmres_tol, or after
 *                gmres_maxit iterations (then SKEL_ENOCONV).
 *  kernel      : SKEL_KERNEL_STOKES (default): the bordered Stokes system
 *                above, 2 DOFs per node, 2N + 3p unknowns.
 *                SKEL_KERNEL_LAPLACE: the Laplace Neumann variant of
 *                Sec. 4.4.1.  Representation u = S mu (single layer), one
 *                DOF per node, N unknowns, no bordering.  Equation
 *                (1/2 I + D + N) mu = g, with g the flux dn u (n out of
 *                Omega), D the normal derivative of S at the target (the
 *                paper's D), and N mu = int mu dy, which completes the
 *                one-dimensional null space of the interior Neumann
 *                problem.  The paper writes the same operator as
 *                -1/2 I - D + N with the data's sign flipped.  FP64 only;
 *                skel_eval_velocity returns the potential u (nt x nrhs).
 *                The Stokes-only calls (point-force data, matvec_df,
 *                adjoint matvec, shape gradients, the no-alloc
 *                evaluation) return SKEL_EINVAL.                         */
typedef struct {
  int32_t leaf_size;
  int32_t n_proxy;
  double proxy_ratio;
  double id_tol;
  int32_t precision;
  double gmres_tol;
  int32_t gmres_maxit;
  int32_t kernel;
} skel_params;

/* Boundary geometry: N trapezoid nodes t_j on p+1 closed curves.
 *  x, y       : gamma(t_j)
 *  dx, dy     : gamma'(t_j)
 *  ddx, ddy   : gamma''(t_j)
 *  dt         : parameter spacing of node j's curve (weight |gamma'| dt)
 *  comp       : 0 for the outer curve Gamma_0 (counter-clockwise), i in
 *               1..p for hole Gamma_i (clockwise)
 *  centers    : p x 2 row-major, c_i strictly inside hole i (Sec. 3.1)   */
typedef struct {
  int64_t N;
  int32_t p;
  const double *x, *y;
  const double *dx, *dy;
  const double *ddx, *ddy;
  const double *dt;
  const int32_t *comp;
  const double *centers;
} skel_geom;

/* Default parameters (leaf 64, 64 proxies at 1.5x, id_tol 1e-12, FP64). */
void skel_default_params(skel_params *out);

/* Build the context: copies the geometry to the device, forms normals,
 * weights and the diagonal curvature term (Sec. 4 opening: trapezoid rule;
 * the diagonal is the smooth limit of the kernel), and builds the quadtree
 * with a fixed root (the bounding square of Gamma_0 with a 1% margin,
 * Sec. 2.8).  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out owns all device state.  Errors: SKEL_EINVAL for N < 1,
 * p < 0, a node outside the root box or a NULL array; SKEL_ENOMEM. */
int skel_build_tree(const skel_geom *geom, const skel_params *params,
                    void *cuda_stream, skel_ctx **out);

/* Factor: recursive skeletonization of -1/2 I + D + N, level by level from
 * the leaves, every box of a level compressed concurrently (Sec. 2.3-2.7),
 * then the bordered top block of Sec. 3.2 (Eq. partition) and its LU.
 * Errors: SKEL_ESINGULAR, SKEL_ECAPACITY, SKEL_ENOMEM, SKEL_ECUDA. */
int skel_factor(skel_ctx *ctx);

/* Fast update after moved nodes (Sec. 2.8): new_geom holds the full new
 * geometry in the same node order (only node_ids[0..n_moved) may differ
 * from the factored one; the hole centres may change).  Only boxes whose
 * compression inputs changed are recompressed; the top block is redone.
 * With the fixed root the result equals a fresh skel_factor of new_geom
 * bit for bit.  Errors as skel_factor, plus SKEL_EINVAL for a node id out of
 * range or a moved node outside the root box. */
int skel_update_moved_nodes(skel_ctx *ctx, int64_t n_moved,
                            const int64_t *node_ids,
                            const skel_geom *new_geom);

/* Fast update after holes were inserted or deleted (Sec. 2.8: the same
 * marking rule as for moved nodes; the paper's insertion and deletion
 * experiments).  new_geom: the full new geometry, whose N and p may differ
 * from the factored one.  old_id[j] (host or device, new_geom->N entries):
 * the node id before the update of new node j, or -1 for a new node.  The
 * ids >= 0 must be increasing, so kept nodes keep their relative order:
 * append inserted holes and remove deleted ones.  Boxes whose subtree
 * holds the same nodes at the same positions, and whose children and near
 * owners are unchanged, keep their factors with their DOF lists
 * renumbered.  The others are recompressed, and the top block (now with
 * the new p's bordering) is redone.  With the fixed root the result equals
 * a fresh skel_factor of new_geom bit for bit.  Errors as skel_factor,
 * plus SKEL_EINVAL for an invalid old_id or a node outside the root box. */
int skel_update_geometry(skel_ctx *ctx, const skel_geom *new_geom,
                         const int64_t *old_id);

/* Solve A [mu; lambda] = [f; g] for nrhs right-hand sides with the factors
 * (Eq. kinv, Eq. solution).  f: (2N+3p) x nrhs, out: same shape (may not
 * alias f).  In SKEL_MIXED form the factored solve preconditions GMRES on
 * the FP64 operator.  Errors: SKEL_ESTATE before skel_factor. */
int skel_solve(skel_ctx *ctx, int32_t nrhs, const double *f, double *out);

/* Solve A^T z = g with the same factors (transposed sweeps, Sec. 2.7 last
 * paragraph): same shapes and errors as skel_solve. */
int skel_solve_adjoint(skel_ctx *ctx, int32_t nrhs, const double *g,
                       double *out);

/* Velocity u = D mu + S alpha + R beta (Eq. completed) at nt targets
 * (tx[i], ty[i]) inside Omega from solutions sol ((2N+3p) x nrhs); u is
 * 2 x nt x nrhs (u[(2*i + a) + 2*nt*r]).  Targets on the boundary are not
 * handled (the kernel is singular there). */
int skel_eval_velocity(skel_ctx *ctx, int32_t nrhs, const double *sol,
                       int64_t nt, const double *tx, const double *ty,
                       double *u);

/* skel_eval_velocity without any memory allocation.  The paper has no
 * counterpart: this is an interface addition.  It is for callers that
 * cannot allocate device memory at the point of the call.  Two examples:
 * a process whose free device memory is held by another allocator (a
 * framework's caching pool, so cudaMalloc would fail), and a latency-bound
 * loop that must not stall the whole device (cudaFree synchronises it).
 * Same arguments, layout and result as skel_eval_velocity, with these
 * differences:
 *  - sol, tx, ty and u must be device (or managed) memory: nothing is
 *    staged.  Host pointers give SKEL_EINVAL.
 *  - The partial sums go to one static device array of 4 MiB
 *    (524288 doubles), built into the library and shared by every call in
 *    the process.  nt * nrhs may be at most 262144; larger sizes give
 *    SKEL_ECAPACITY with a message stating the limit.
 *  - nrhs may be at most 65535 (SKEL_EINVAL beyond).
 *  - The first call on each device, and again the first call after the
 *    device's context changes (a device reset, say), looks up that array's
 *    address (cudaGetSymbolAddress, with the device current).  With lazy
 *    module loading that first call may also load the library's device
 *    code, which takes some device memory: make it while memory is still
 *    free, before handing the memory to another allocator, and before any
 *    stream capture begins.
 *  - Calls whose kernels overlap on the GPU race on the shared array (two
 *    threads, contexts or streams); serialise them.  Nothing in the array
 *    needs to start at zero, since every partial sum a call reads it has
 *    written first.
 *  - Runs on the context's stream and waits for it before returning.
 * Errors: SKEL_EINVAL, SKEL_ECAPACITY, SKEL_ECUDA. */
int skel_eval_velocity_noalloc(skel_ctx *ctx, int32_t nrhs, const double *sol,
                               int64_t nt, const double *tx, const double *ty,
                               double *u);

/* Boundary data from point forces (Stokeslets of Sec. 3.1):
 * f = [sum_s S(x_j, s) F_s ; 0] for every node, nrhs sets of ns forces;
 * src_xy, src_f: nrhs x ns x 2.  holes_zero != 0 keeps the data on Gamma_0
 * only (no-slip holes).  f: (2N+3p) x nrhs. */
int skel_point_force_rhs(skel_ctx *ctx, int32_t nrhs, int32_t ns,
                         const double *src_xy, const double *src_f,
                         int32_t holes_zero, double *f);

/* A [mu; lambda] with the FP64 operator, O(N^2) on the fly (the residual
 * used by the refinement).  x, y: (2N+3p) x nrhs.  The partial sums need
 * about 2 KB per node and column; the columns are processed in batches
 * whose scratch stays within 4 GiB. */
int skel_matvec(skel_ctx *ctx, int32_t nrhs, const double *x, double *y);

/* A [mu; lambda] like skel_matvec, with the O(N^2) double-layer sums in
 * double-float arithmetic (pairs of floats, about 48 significant bits, on
 * the FP32 units) and every O(N) term in FP64: relative accuracy about
 * 1e-13 at a fraction of the FP64 cost.  It is the operator of the GMRES
 * iterations of the SKEL_MIXED forward solve (see "gmres_fp64_check" for
 * which residual decides convergence).  Accuracy assumes each curve's
 * nodes are given in order along it.  x, y: (2N+3p) x nrhs. */
int skel_matvec_df(skel_ctx *ctx, int32_t nrhs, const double *x, double *y);

/* A^T z with the FP64 operator (the convergence test of the adjoint solve
 * in SKEL_MIXED form).  z, y: (2N+3p) x nrhs. */
int skel_matvec_adjoint(skel_ctx *ctx, int32_t nrhs, const double *z,
                        double *y);

/* A^T z like skel_matvec_adjoint, with the O(N^2) double-layer sums in
 * double-float arithmetic as in skel_matvec_df: the operator of the GMRES
 * iterations of the SKEL_MIXED adjoint solve.  z, y: (2N+3p) x nrhs. */
int skel_matvec_adjoint_df(skel_ctx *ctx, int32_t nrhs, const double *z,
                           double *y);

/* Shape derivatives (the differentiation path).  The paper's shape
 * optimisation (Sec. 4.3) estimates gradients by finite differences and
 * points to adjoint methods for larger problems; these two calls give the
 * pieces of the adjoint gradient.  The geometry gradient layout g is that
 * of skel_geom's differentiated arrays: 6N values d/dx, d/dy, d/ddx...
 * in the order x, y, dx, dy, ddx, ddy (N each, the samples gamma, gamma',
 * gamma''), then 2p values d/dcenters (p x 2, row-major); dt and comp are
 * not differentiated.  All arrays may be host or device memory.
 *
 * For J(geometry) = sum_t |u(x_t)|^2 with u = E s, A s = f (f independent
 * of the differentiated samples, e.g. no-slip holes moved against a fixed
 * outer curve):  ubar = 2u;  skel_grad_velocity -> (gs, gE);
 * skel_solve_adjoint(gs) -> z;  skel_grad_bilinear(z, s) -> gA;
 * dJ/dgeometry = gE - gA. */

/* The shape-optimisation objective of the paper's Sec. 4.3 setting in one
 * call each, value and gradient (Stokes form; f must not depend on the
 * differentiated samples, e.g. point-force data on a fixed outer curve and
 * no-slip holes):
 *  skel_velocity_energy: s = A^{-1} f (factored solve, or GMRES in the
 *    SKEL_MIXED form) and J = sum_t |u(tx_t, ty_t)|^2 with u the velocity
 *    (Eq. completed) at nt interior targets.  f, s: (2N+3p); *J: one
 *    double (host or device).
 *  skel_velocity_energy_gradient: g = dJ/dgeometry (layout of
 *    skel_grad_bilinear: 6N + 2p doubles) at that solution s, by the
 *    adjoint method: ubar = 2u, (gs, gE) = skel_grad_velocity,
 *    A^T z = gs (skel_solve_adjoint), gA = skel_grad_bilinear(z, s),
 *    g = gE - gA.  Needs the factorization of the same geometry.
 * Errors: SKEL_EINVAL, SKEL_ESTATE (before skel_factor), SKEL_ENOCONV (a
 * mixed-form GMRES), SKEL_ECUDA. */
int skel_velocity_energy(skel_ctx *ctx, const double *f, int64_t nt,
                         const double *tx, const double *ty, double *J,
                         double *s);
int skel_velocity_energy_gradient(skel_ctx *ctx, const double *s, int64_t nt,
                                  const double *tx, const double *ty,
                                  double *g);

/* g = d/dgeometry of L = z^T A(geometry) s for fixed z, s ((2N+3p) each):
 * the stresslet pairs, the diagonal limit, N, H and Psi terms of A. */
int skel_grad_bilinear(skel_ctx *ctx, const double *z, const double *s,
                       double *g);

/* For the velocity at nt interior targets (tx, ty held fixed) and weights
 * ubar (2 x nt, the layout of skel_eval_velocity's u): gs = E^T ubar
 * ((2N+3p)) and g = d/dgeometry of ubar . E(geometry) s (layout above). */
int skel_grad_velocity(skel_ctx *ctx, const double *s, int64_t nt,
                       const double *tx, const double *ty, const double *ubar,
                       double *gs, double *g);

/* Tuning parameters of the launch shapes (integers; defaults in
 * parentheses).  They change no arithmetic of the method, only which
 * kernel runs a box and how work is cut into CTAs:
 *   "cluster_min_n" (max(160, 1.25 x DOFs per node x leaf_size)): boxes
 *       with at least this many active DOFs are compressed and eliminated
 *       by 16-CTA clusters;
 *   "cluster_level_boxes" (76): on levels with at most this many boxes,
 *       every box with more active DOFs than two leaves goes to the
 *       clusters as well;
 *   "sweep_rhs_chunk" (16): right-hand sides per CTA in the level sweeps
 *       (4, 8 or 16);
 *   "cluster_mid_min_n" (off: 2^30) and "cluster_mid_level_boxes" (304):
 *       boxes that are not large but have at least cluster_mid_min_n
 *       active DOFs, on levels of at most cluster_mid_level_boxes boxes,
 *       go to 4-CTA clusters;
 *   "wide_min_n" (256): cluster-class boxes with at least this many active
 *       DOFs are eliminated by a sequence of launches that each spread
 *       over the whole GPU (tiled GEMMs for Eq. tmat / schurmat, a
 *       blocked LU of X_RR and blocked triangular solves; up to four such
 *       boxes at once on their own streams) instead of one cluster (FP64
 *       factors only);
 *   "wide_qr_min_n" (1024): of those, boxes with at least this many active
 *       DOFs, on levels with at least two such boxes, also run their
 *       column-pivoted QR as one-CTA pivot steps and reflector
 *       applications over the whole GPU;
 *   "tc_products" (0): in the SKEL_MIXED form, 1 runs those boxes'
 *       products of Eq. tmat / Eq. schurmat (X_RS, X_SR, X_RR, X_SS) on
 *       the tensor cores in 3xTF32 (see skel_gemm_tf32x3); the LU of
 *       X_RR and the triangular solves stay FP64.
 * Setting one drops the factorization (SKEL_ESTATE until skel_factor runs
 * again), so factors and updates always come from one set of launch
 * shapes.  One more key is a solve setting and keeps the factors:
 *   "gmres_fp64_check" (0): in the SKEL_MIXED form, 1 decides GMRES
 *       convergence on the FP64 operator's residual always; with 0 the
 *       double-float operator's residual decides it when gmres_tol >=
 *       1e-11 (its relative accuracy is about 2e-13) and the FP64 one
 *       below that.  The double-float test reads the residual of a cycle
 *       that met a quarter of gmres_tol from the GMRES recurrence (the
 *       Arnoldi relation of that operator, no further apply; stats key
 *       gmres_recurrence = 1); the FP64 test applies the FP64 operator.
 * Errors: SKEL_EINVAL for an unknown key or value.  The Python module
 * paper_2001_11619_gb300.autotune searches the launch shapes on a
 * workload. */
int skel_set_tuning(skel_ctx *ctx, const char *key, double value);
int skel_get_tuning(skel_ctx *ctx, const char *key, double *value);

/* Per-kernel device timing.  on != 0 records a CUDA event pair around
 * every kernel launch group on the context's stream and accumulates, per
 * kernel, the launch count, the device time and the algorithmic flop and
 * byte counts; skel_stats reports them under "kernels".  Each call resets
 * the accumulators.  Timing adds a little host overhead per launch group. */
int skel_set_timing(skel_ctx *ctx, int32_t on);

/* Device memory: the library keeps the blocks that contexts free (factor
 * arenas, bordered columns, scratch) in a process-wide cache per device
 * and reuses them for later requests of at most their size and at least
 * half of it, so that building many solvers does not pay cudaMalloc and
 * cudaFree (which synchronises the device) each time.  The cache holds at
 * most half of the device memory (environment SKEL_CACHE_LIMIT_GB
 * overrides it at the first release; 0 disables caching); a failing
 * allocation empties it and retries.  This call returns every cached
 * block to the driver (all devices).  Returns SKEL_OK or SKEL_ECUDA. */
int skel_release_cached_memory(void);

/* Measured arithmetic peaks of the current device (no counterpart in the
 * paper; the denominators of the roofline fractions of the ALU-bound
 * kernels).  A kernel of independent fused multiply-add chains over every
 * SM is timed with CUDA events on the legacy default stream, after a
 * warm-up launch: out[0] = FP64 and out[1] = FP32 FMA throughput in
 * TFLOP/s (2 flops per FMA).  Takes about 0.2 s; synchronous.  Errors:
 * SKEL_EINVAL (out NULL), SKEL_ENOMEM, SKEL_ECUDA. */
int skel_measure_alu_peaks(double *out);

/* C = C - A B in split precision on the tensor cores (no counterpart in
 * the paper; the building block of the SKEL_MIXED form's large-box
 * products of Eq. tmat / Eq. schurmat, exposed for its parity test).
 * Column-major FP64 device arrays: A is M x K (lda >= M), B is K x N
 * (ldb >= K), C is M x N (ldc >= M).  Each entry is rounded to FP32 and
 * split into two TF32 parts; three TF32 products per pair accumulate in
 * FP32 (tcgen05.mma kind::tf32), so the result has about FP32 accuracy:
 * |error| <= about K 2^-22 (|A| |B|) entrywise.  Runs on `stream` and
 * waits for it.  Errors: SKEL_EINVAL (sizes or strides), SKEL_ENOMEM,
 * SKEL_ETIMEOUT (a tensor-core wait ran out), SKEL_ECUDA. */
int skel_gemm_tf32x3(int32_t M, int32_t N, int32_t K, const double *A,
                     int64_t lda, const double *B, int64_t ldb, double *C,
                     int64_t ldc, void *stream);

/* Number of kernels launched by this library in this process so far. */
int64_t skel_kernel_launches(void);

/* JSON summary (levels, boxes, ranks per level, timings, flop and byte
 * counts of the last factor/solve) written into json[0..cap).  In the
 * SKEL_MIXED form it also gives the GMRES iterations and final relative
 * residual of the last solve (largest over its columns) and the relative
 * residual after the preconditioner alone (gmres_relres0, last column);
 * gmres_check ("df" or "fp64") names the operator whose residual decided
 * convergence, and gmres_recurrence = 1 when that residual was read from
 * the GMRES recurrence (see "gmres_fp64_check" at skel_set_tuning).
 * host_factor_ms / host_update_ms / host_solve_ms: wall time of the last
 * such call minus the time it spent blocked in stream synchronisations,
 * i.e. the host's own bookkeeping (index lists, tree, marking), during
 * which the GPU idles when nothing is queued.  host_prep_ms / host_post_ms:
 * the part of it spent in the level loop before each level's launches
 * (active and near-field lists, sizes, uploads) and after its read-back,
 * summed over the levels of the last factor or update. */
int skel_stats(skel_ctx *ctx, char *json, size_t cap);

/* Last error message of ctx (or of the last failed skel_build_tree when
 * ctx is NULL). */
const char *skel_last_error(skel_ctx *ctx);

void skel_destroy(skel_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SKEL_H */
