// Host runtime of the skeletonization solver and the C ABI of skel.h.
//
// The host keeps the quadtree and the index bookkeeping (active-DOF lists,
// proxy-disk near fields, factor offsets); every floating-point step of
// the factorization and of the solves runs in the CUDA kernels.  One level
// of the tree is one batch of kernel launches over all its boxes
// (Sec. 2.7: boxes of a level are compressed concurrently from the
// start-of-level state).
#include <algorithm>
#include <type_traits>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "skel_internal.h"

using namespace skel;

#include <atomic>

namespace {

std::string g_last_error;
std::atomic<int64_t> g_launches{0};

// kernel groups reported by the timing mode
enum KCat {
  KC_QUAD,
  KC_DIAG,
  KC_IDMAT,
  KC_CPQR,
  KC_ELIM,
  KC_BORDER,
  KC_GRAM,
  KC_TOPLU,
  KC_UP,
  KC_DOWN,
  KC_TOPSOLVE,
  KC_EVAL,
  KC_RHS,
  KC_MATVEC,
  KC_MATVEC_DF,
  KC_GRAD,
  KC_N
};
const char *kKcName[KC_N] = {
    "quadrature", "assemble_diag", "assemble_id", "cpqr",
    "eliminate",  "bordered_sweeps", "gram",      "top_lu",
    "solve_up",   "solve_down",    "solve_top",   "eval_velocity",
    "point_force_rhs", "matvec", "matvec_df", "shape_gradient"};

struct KStat {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

// FP64 operations counted per evaluated stresslet entry (differences,
// squared distance, normal projection, one division, scaling, outer
// product): the unit of the assembly and evaluation work counts.
constexpr double kEntryFlops = 16.0;
// flops per source-target pair of the operator and evaluation sums: the
// 2 x 2 stresslet block formed and applied to a two-component density
// (difference 2, |r|^2 3, 1/|r|^4 2, r.n 3, coefficient 2, block 6,
// block times density 6, accumulation 2, weight and scaling 4).  The
// kernels exploit the block's rank-one form and issue 16 FP64
// instructions (24 flops) per pair.
constexpr double kPairFlops = 30.0;
// GMRES tolerances at or above this decide convergence on the double-float
// residual (relative accuracy about 2e-13, so a 1e-11 test keeps 50x room)
constexpr double kDfCheckTol = 1e-11;
// columns (right-hand sides) per call: one grid row per column in several
// launches (CUDA's grid y limit)
constexpr int kMaxCols = 65535;
// concurrent streams of the whole-GPU elimination of the wide boxes
constexpr int kWideStreams = 4;
// scratch budget of the operator's partial sums in skel_matvec
constexpr size_t kMatvecScratchBytes = (size_t)4 << 30;

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { dev_free(p); }
  cudaError_t ensure(size_t cnt) {
    if (cnt <= n && p) return cudaSuccess;
    dev_free(p);
    p = nullptr;
    n = 0;
    void *q = nullptr;
    cudaError_t e = dev_alloc(&q, std::max<size_t>(cnt, 1) * sizeof(T));
    p = static_cast<T *>(q);
    if (e == cudaSuccess) n = std::max<size_t>(cnt, 1);
    return e;
  }
};

// Growable device arena: offsets stay valid when it grows.
template <class T>
struct Arena {
  T *p = nullptr;
  int64_t cap = 0, used = 0;
  Arena() = default;
  Arena(const Arena &) = delete;
  ~Arena() { dev_free(p); }
  bool fits(int64_t cnt) const { return used + (cnt + 31) / 32 * 32 <= cap; }
  cudaError_t alloc(int64_t cnt, cudaStream_t s, int64_t &off) {
    cnt = (cnt + 31) / 32 * 32;
    if (used + cnt > cap) {
      int64_t nc = std::max<int64_t>({2 * cap, used + cnt, (int64_t)1 << 20});
      void *q = nullptr;
      cudaError_t e = dev_alloc(&q, nc * sizeof(T));
      if (e != cudaSuccess) return e;
      T *np = static_cast<T *>(q);
      if (p) {
        cudaMemcpyAsync(np, p, used * sizeof(T), cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
        dev_free(p);
      }
      p = np;
      cap = nc;
    }
    off = used;
    used += cnt;
    return cudaSuccess;
  }
};

struct Status {
  int code = SKEL_OK;
  std::string msg;
};

// One factorization's bordered sweeps (Sec. 3.2), level by level
struct BordState {
  bool on = false;
  bool full_b = true;      // every box gets a new snapshot (and is swept)
  bool full = false;       // everything is swept from the current level up
  bool prev_full = false;  // the level below was swept completely
  const std::vector<char> *dirty = nullptr;  // recompressed boxes
  std::vector<int> lv_q;                     // chunk width per level
  std::vector<char> col_prev;  // H columns swept on the level below
  int64_t off = 0;             // next free int of the item buffer
};

}  // namespace

struct skel_ctx {
  skel_params prm{};
  cudaStream_t st = nullptr;
  // factorizations and updates run on sthi, a stream of the highest
  // priority forked from the caller's stream (ev_in) and joined back
  // (ev_out): their level-by-level compression is the critical path, and
  // the bordered sweeps on st3 (lowest priority) fill the SMs it leaves
  cudaStream_t sthi = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int64_t N = 0;
  int p = 0;
  std::string err;
  // host copies of the raw geometry (tree building, near fields, update
  // change detection)
  std::vector<double> hx, hy, hdx, hdy, hddx, hddy, hdt, hcent;
  std::vector<int32_t> hcomp;
  double root_cx = 0, root_cy = 0, root_hw = 0;
  // device geometry
  DBuf<double> gx, gy, gdx, gdy, gddx, gddy, gdt, gnx, gny, gw, gkap, gcent;
  DBuf<int32_t> gcomp;
  std::vector<int32_t> hdlf_blk;  // double-float operator target blocks
  DBuf<int32_t> dlf_blk;
  DBuf<double> dlfscr;
  DBuf<double> gscr;  // shape-derivative partial sums
  DBuf<float> gf32;  // float copies: xh, xl, yh, yl, nx, ny, w, kap
  DevGeom g{};
  Tree tree;
  // factors
  bool factored = false;
  std::vector<DevBox> hbox;
  std::vector<std::vector<int32_t>> hdofs;  // skeleton first, then redundant
  std::vector<std::vector<int>> hnear;      // near owners at the box's level
  std::vector<uint64_t> content;            // subtree content digest
  DBuf<DevBox> dbox;
  Arena<double> fac;
  Arena<int32_t> ipool, dofs;
  int64_t live_fac = 0;
  // per-level scratch
  DBuf<LvlBox> dlb;
  DBuf<int32_t> iscr;
  DBuf<int32_t> dflag, dmoves, dfsel;  // X_RR conditioning moves per level
  DBuf<double> dscr;   // ID matrices and diagonal blocks (storage type)
  DBuf<double> tws;    // FP64 workspace for the interpolation matrices T
  DBuf<double> dsa;    // diagonal blocks (factor type)
  bool id32 = false;   // ID matrices in FP32 (mixed form)
  bool fac32 = false;  // factors in FP32 (mixed form with FP32 elimination)
  DBuf<int> dstatus;
  DBuf<int32_t> lvl_ids;
  std::vector<int64_t> lvl_off;
  // root and bordered data (Sec. 3.2)
  std::vector<int32_t> root_act;
  int s = 0, ldt = 0;
  DBuf<int32_t> droot_act, top_piv;
  DBuf<uint8_t> rmask;
  DBuf<double> UH, W, QT, Wt, G, top, partial;
  // solve scratch
  DBuf<double> work, rhs_top, vin, vout, dlscr;
  // refinement (mixed form): Krylov basis, preconditioned basis, scratch
  DBuf<double> gmV, gmZ, gmw, gmdot, gmx;
  bool gmres_fp64_check = false;  // always decide convergence in FP64
  // whole-GPU elimination of boxes with at least wide_min_n active DOFs
  int wide_min_n = 256;
  int wide_qr_min_n = 1024;  // and of at least this many, the CPQR too
  // mixed form: the wide boxes' products on the tensor cores (3xTF32)
  bool tc_products = false;
  DBuf<double> wkp, wxs;
  DBuf<int32_t> wiws;
  // wide boxes of one level run on up to kWideStreams streams at once
  cudaStream_t wst[kWideStreams] = {};
  cudaEvent_t wev[kWideStreams] = {}, wev_fork = nullptr;
  // the wide boxes' CPQR: descriptors, norms, permutations, R11 in FP64,
  // and pinned stop flags with their events
  DBuf<char> qops;
  DBuf<double> qdws, qR;
  DBuf<int32_t> qiws;
  volatile int32_t *qr_hstop = nullptr;
  std::vector<cudaEvent_t> qr_events;
  DBuf<int32_t> gscr_i;  // chunk lists of the sparse Gram product
  DBuf<double> escr;     // velocity-energy value and gradient
  DBuf<char> wops;
  bool last_check_df = false;     // the last solve's test was double-float
  bool last_check_rec = false;    // ... on the GMRES residual recurrence
  int last_iters = 0;
  double last_relres = 0.0, last_relres0 = 0.0;
  // statistics
  double t_factor_ms = 0, t_solve_ms = 0, t_update_ms = 0;
  // time blocked in stream synchronisations, and the host's own share
  // (wall minus blocked) of the last factor / update / solve call
  double alloc_ms = 0;  // device allocation time of the last factor / update
  double wait_ms = 0, host_factor_ms = 0, host_update_ms = 0,
         host_solve_ms = 0;
  // host time of the level loop before each level's launches (lists,
  // sizes, uploads) and after its read-back, summed over the levels
  double host_prep_ms = 0, host_post_ms = 0;
  int64_t last_dirty = 0, last_boxes = 0;
  std::vector<int> lv_nbox, lv_maxn, lv_maxk, lv_maxm, lv_big, lv_moved,
      lv_wide;
  std::vector<int> lv_alln;  // largest box of each level (all boxes)
  std::vector<double> lv_ms;
  double flops_factor = 0;
  // auxiliary stream for the cluster kernels of large boxes
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // tuning parameters (skel_set_tuning): boxes with at least
  // cluster_min_n active DOFs, and on levels of at most cluster_level_boxes
  // boxes every box larger than two leaves, go to the cluster kernels;
  // sweep_rhs_chunk caps the right-hand sides per CTA of the sweeps
  int cluster_min_n = 160;
  int cluster_level_boxes = 76;
  // mid-size boxes (4-CTA clusters): at least cluster_mid_min_n active DOFs
  // on levels of at most cluster_mid_level_boxes boxes
  int cluster_mid_min_n = 1 << 30;
  int cluster_mid_level_boxes = 304;
  int sweep_rhs_chunk = 16;
  // timing mode
  bool timing = false;
  // Bordered sweeps (Sec. 3.2): the initial columns H0 = H, P0 = Psi, the
  // arena of per-box b_S snapshots (DevBox::snap_off), and for the next
  // factor_top which H columns changed everywhere (a moved hole's centre)
  // or whether everything is swept again (bord_full)
  Arena<double> snap;
  DBuf<double> H0, P0;
  DBuf<int32_t> sitems;
  // the sweeps run on their own stream (st3), level by level as soon as a
  // level's factors exist, beside the compression of the levels above;
  // they read their own copy of the box records and report into dstatus3
  cudaStream_t st3 = nullptr;
  cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
  DBuf<DevBox> dbox_sw;
  DBuf<int> dstatus3;
  BordState bs;
  // pinned staging for st3's uploads (a copy from pageable memory may wait
  // for the stream); regions are handed out once per factorization
  char *pin = nullptr;
  size_t pin_cap = 0, pin_used = 0;
  std::vector<char> bord_col_changed;
  bool bord_full = true;
  std::vector<int> bord_lv_q;  // chunk width per level of the last sweep
  // kernel family: Laplace Neumann form (1 DOF per node, no bordering) or
  // Stokes (2 DOFs per node, 3p bordering columns)
  bool lap = false;
  int dpn = 2;
  // Single right-hand-side factored solves (the GMRES preconditioner and
  // one-column solves) replayed from a CUDA graph per direction (index:
  // adjoint), captured on the first such solve after a factorization or
  // update; gsol is the graph's fixed column.
  bool graphs = true;
  cudaGraphExec_t sgraph[2] = {nullptr, nullptr};
  int64_t sgraph_launches[2] = {0, 0};
  DBuf<double> gsol;
  KStat kst[KC_N];
  // (category | level << 8, event pair) of timed launch groups
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  int cur_level = 0;  // level being compressed (0: none)
  std::vector<std::vector<double>> lv_kms;  // per level, ms per category
  // timings recorded on st3, folded in once st3 is known to be done
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending3;
  std::vector<cudaEvent_t> evpool;
  ~skel_ctx() {
    for (auto &p : pending) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    for (auto &p : pending3) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    if (st3) cudaStreamSynchronize(st3);
    if (pin) cudaFreeHost(pin);
    if (ev_fork3) cudaEventDestroy(ev_fork3);
    if (ev_join3) cudaEventDestroy(ev_join3);
    if (st3) cudaStreamDestroy(st3);
    for (auto e : evpool) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    for (auto &g : sgraph)
      if (g) cudaGraphExecDestroy(g);
    if (st2) cudaStreamDestroy(st2);
    if (sthi) cudaStreamDestroy(sthi);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    for (int i = 0; i < kWideStreams; ++i) {
      if (wst[i]) cudaStreamDestroy(wst[i]);
      if (wev[i]) cudaEventDestroy(wev[i]);
    }
    if (wev_fork) cudaEventDestroy(wev_fork);
    for (auto e : qr_events) cudaEventDestroy(e);
    if (qr_hstop) cudaFreeHost((void *)qr_hstop);
  }
};

void skel::note_launches(int n) { g_launches += n; }

// DOF counts: density DOFs (dpn per node), bordering unknowns (3 per hole
// for Stokes, none for Laplace) and their sum, the leading dimension of
// every right-hand side and solution column
static int64_t ndof(const skel_ctx *c) { return (int64_t)c->dpn * c->N; }
static int nbord(const skel_ctx *c) { return c->lap ? 0 : 3 * c->p; }
static int64_t nsys(const skel_ctx *c) { return ndof(c) + nbord(c); }
static int64_t dof_node(const skel_ctx *c, int64_t d) {
  return c->dpn == 2 ? d >> 1 : d;
}

static int fail(skel_ctx *ctx, int code, const std::string &msg);
static int stokes_only(skel_ctx *ctx) {
  return fail(ctx, SKEL_EINVAL, "not available for the Laplace form");
}

static void drop_graphs(skel_ctx *ctx) {
  for (int a = 0; a < 2; ++a) {
    if (ctx->sgraph[a]) cudaGraphExecDestroy(ctx->sgraph[a]);
    ctx->sgraph[a] = nullptr;
  }
}

static cudaEvent_t get_event(skel_ctx *c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Run one kernel launch group of category `cat`; with timing on, bracket it
// with events on the context's stream.
template <class F>
static void timed(skel_ctx *c, int cat, F &&f) {
  const int64_t l0 = g_launches.load();
  if (!c->timing) {
    f();
    c->kst[cat].launches += g_launches.load() - l0;
    return;
  }
  cudaEvent_t a = get_event(c), b = get_event(c);
  cudaEventRecord(a, c->st);
  f();
  cudaEventRecord(b, c->st);
  c->pending.push_back({cat | (c->cur_level << 8), {a, b}});
  c->kst[cat].launches += g_launches.load() - l0;
}

// As timed(), on another stream; resolved by resolve_timing3 once that
// stream is known to be done.
template <class F>
static void timed_on(skel_ctx *c, int cat, cudaStream_t st, F &&f) {
  const int64_t l0 = g_launches.load();
  if (!c->timing) {
    f();
    c->kst[cat].launches += g_launches.load() - l0;
    return;
  }
  cudaEvent_t a = get_event(c), b = get_event(c);
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  c->pending3.push_back({cat, {a, b}});
  c->kst[cat].launches += g_launches.load() - l0;
}

static void resolve_timing3(skel_ctx *c) {
  for (auto &p : c->pending3) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) ==
        cudaSuccess)
      c->kst[p.first].ms += ms;
    c->evpool.push_back(p.second.first);
    c->evpool.push_back(p.second.second);
  }
  c->pending3.clear();
}

// After a stream synchronisation: fold the recorded event pairs in.
static void resolve_timing(skel_ctx *c) {
  for (auto &p : c->pending) {
    float ms = 0.f;
    const int cat = p.first & 255, lev = p.first >> 8;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) ==
        cudaSuccess) {
      c->kst[cat].ms += ms;
      if (lev > 0 && lev < (int)c->lv_kms.size()) c->lv_kms[lev][cat] += ms;
    }
    c->evpool.push_back(p.second.first);
    c->evpool.push_back(p.second.second);
  }
  c->pending.clear();
}

#define CU(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess)                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SKEL_ENOMEM      \
                                                       : SKEL_ECUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

static int fail(skel_ctx *ctx, int code, const std::string &msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_last_error = msg;
  return code;
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch())
      .count();
}

// stream synchronisation that books the time the host spends blocked on
// the GPU, so that wall time minus this is the host's own share
static cudaError_t sync_st(skel_ctx *ctx) {
  const double t0 = now_ms();
  const cudaError_t e = cudaStreamSynchronize(ctx->st);
  ctx->wait_ms += now_ms() - t0;
  return e;
}

// Digests of every box's subtree content (node ids and raw geometry), for
// the update's change test: a leaf mixes its nodes' words, an internal box
// mixes its children's digests (children have larger ids than their
// parent, so one backward pass suffices and each node is read once).
static inline uint64_t mix64(uint64_t h, uint64_t w) {
  h ^= w * 0x9E3779B97F4A7C15ull;
  h = (h << 27) | (h >> 37);
  return h * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
}

// ident: the identity hashed for node j (nullptr: j itself).  An update
// that renumbers nodes hashes their ids before the update, so that a box
// whose nodes only changed number keeps its digest.
static void box_contents(skel_ctx *ctx, const int64_t *ident = nullptr) {
  const Tree &t = ctx->tree;
  const size_t nb = t.boxes.size();
  ctx->content.assign(nb, 0);
  for (size_t q = nb; q-- > 0;) {
    const HBox &B = t.boxes[q];
    uint64_t h = 0x243F6A8885A308D3ull ^ (uint64_t)B.leaf;
    if (B.leaf) {
      for (int64_t i = B.nbeg; i < B.nbeg + B.ncnt; ++i) {
        const int64_t j = ctx->tree.order[i];
        const double v[7] = {ctx->hx[j],  ctx->hy[j],   ctx->hdx[j],
                             ctx->hdy[j], ctx->hddx[j], ctx->hddy[j],
                             ctx->hdt[j]};
        uint64_t w[7];
        std::memcpy(w, v, sizeof w);
        h = mix64(h, (uint64_t)(ident ? ident[j] : j));
        for (int u = 0; u < 7; ++u) h = mix64(h, w[u]);
      }
    } else {
      for (int c = 0; c < B.nchild; ++c)
        h = mix64(h, ctx->content[B.child[c]]);
    }
    ctx->content[q] = mix64(h, (uint64_t)B.ncnt);
  }
}

static void node_dofs(const skel_ctx *ctx, const HBox &B,
                      std::vector<int32_t> &out) {
  out.clear();
  // nodes of a box are ascending ids inside Tree::order
  for (int64_t i = B.nbeg; i < B.nbeg + B.ncnt; ++i) {
    int64_t j = ctx->tree.order[i];
    if (ctx->dpn == 1) {
      out.push_back((int32_t)j);
    } else {
      out.push_back((int32_t)(2 * j));
      out.push_back((int32_t)(2 * j + 1));
    }
  }
}

static void level_act(const skel_ctx *ctx, int b, std::vector<int32_t> &out) {
  const HBox &B = ctx->tree.boxes[b];
  if (B.leaf) {
    node_dofs(ctx, B, out);
    return;
  }
  out.clear();
  for (int c = 0; c < B.nchild; ++c) {
    int cb = B.child[c];
    const auto &d = ctx->hdofs[cb];
    out.insert(out.end(), d.begin(), d.begin() + ctx->hbox[cb].k);
  }
}

// Upload geometry (host or device source) and form the quadrature.
static int load_geometry(skel_ctx *ctx, const skel_geom *geom) {
  const int64_t N = geom->N;
  const int p = geom->p;
  auto up = [&](DBuf<double> &d, std::vector<double> &h, const double *src,
                int64_t cnt) -> cudaError_t {
    cudaError_t e = d.ensure(cnt);
    if (e != cudaSuccess) return e;
    h.resize(cnt);
    if (cnt == 0) return cudaSuccess;
    e = cudaMemcpy(h.data(), src, cnt * sizeof(double), cudaMemcpyDefault);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(d.p, h.data(), cnt * sizeof(double),
                           cudaMemcpyHostToDevice, ctx->st);
  };
  CU(up(ctx->gx, ctx->hx, geom->x, N));
  CU(up(ctx->gy, ctx->hy, geom->y, N));
  CU(up(ctx->gdx, ctx->hdx, geom->dx, N));
  CU(up(ctx->gdy, ctx->hdy, geom->dy, N));
  CU(up(ctx->gddx, ctx->hddx, geom->ddx, N));
  CU(up(ctx->gddy, ctx->hddy, geom->ddy, N));
  CU(up(ctx->gdt, ctx->hdt, geom->dt, N));
  CU(up(ctx->gcent, ctx->hcent, geom->centers, 2 * (int64_t)p));
  CU(ctx->gcomp.ensure(N));
  ctx->hcomp.resize(N);
  CU(cudaMemcpy(ctx->hcomp.data(), geom->comp, N * sizeof(int32_t),
                cudaMemcpyDefault));
  for (int64_t i = 0; i < N; ++i)
    if (ctx->hcomp[i] < 0 || ctx->hcomp[i] > p)
      return fail(ctx, SKEL_EINVAL, "comp out of range at node " +
                                        std::to_string(i));
  for (int64_t i = 0; i < N; ++i)
    if (!(ctx->hdx[i] * ctx->hdx[i] + ctx->hdy[i] * ctx->hdy[i] > 0) ||
        !(ctx->hdt[i] > 0) || !std::isfinite(ctx->hx[i]) ||
        !std::isfinite(ctx->hy[i]))
      return fail(ctx, SKEL_EINVAL,
                  "degenerate or non-finite node " + std::to_string(i));
  CU(cudaMemcpyAsync(ctx->gcomp.p, ctx->hcomp.data(), N * sizeof(int32_t),
                     cudaMemcpyHostToDevice, ctx->st));
  // target blocks of the double-float operator: runs of consecutive nodes of
  // one curve, at most dlf_block_size() long (compact arcs when each curve's
  // nodes are given in order along it)
  ctx->hdlf_blk.clear();
  for (int64_t i = 0; i < N;) {
    int64_t e = i + 1;
    while (e < N && e - i < dlf_block_size() && ctx->hcomp[e] == ctx->hcomp[i])
      ++e;
    ctx->hdlf_blk.push_back((int32_t)i);
    ctx->hdlf_blk.push_back((int32_t)(e - i));
    i = e;
  }
  CU(ctx->dlf_blk.ensure(ctx->hdlf_blk.size()));
  CU(cudaMemcpyAsync(ctx->dlf_blk.p, ctx->hdlf_blk.data(),
                     ctx->hdlf_blk.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, ctx->st));
  CU(ctx->gnx.ensure(N));
  CU(ctx->gny.ensure(N));
  CU(ctx->gw.ensure(N));
  CU(ctx->gkap.ensure(N));
  CU(ctx->gf32.ensure(8 * (size_t)N));
  timed(ctx, KC_QUAD, [&] {
    launch_quadrature(ctx->gx.p, ctx->gy.p, ctx->gdx.p, ctx->gdy.p,
                      ctx->gddx.p, ctx->gddy.p, ctx->gdt.p, N, ctx->gnx.p,
                      ctx->gny.p, ctx->gw.p, ctx->gkap.p, ctx->gf32.p,
                      ctx->st);
  });
  CU(cudaGetLastError());
  ctx->N = N;
  ctx->p = p;
  DevGeom &g = ctx->g;
  g.N = N;
  g.p = p;
  g.lap = ctx->lap ? 1 : 0;
  g.x = ctx->gx.p;
  g.y = ctx->gy.p;
  g.nx = ctx->gnx.p;
  g.ny = ctx->gny.p;
  g.w = ctx->gw.p;
  g.kap = ctx->gkap.p;
  g.comp = ctx->gcomp.p;
  g.centers = ctx->gcent.p;
  const float *f = ctx->gf32.p;
  g.xh = f;
  g.xl = f + N;
  g.yh = f + 2 * N;
  g.yl = f + 3 * N;
  g.nxf = f + 4 * N;
  g.nyf = f + 5 * N;
  g.wf = f + 6 * N;
  g.kapf = f + 7 * N;
  return SKEL_OK;
}

static int check_geom_args(const skel_geom *geom) {
  if (!geom || geom->N < 1 || geom->p < 0 || !geom->x || !geom->y ||
      !geom->dx || !geom->dy || !geom->ddx || !geom->ddy || !geom->dt ||
      !geom->comp || (geom->p > 0 && !geom->centers))
    return SKEL_EINVAL;
  if (geom->N > (int64_t)1 << 29) return SKEL_EINVAL;  // 32-bit DOF ids
  return SKEL_OK;
}

// ---------------------------------------------------------------------------
// precision of the factors: FP64, or float in the mixed form.  The factor
// pool and the level scratch are allocated in doubles and addressed in
// units of the storage type.

static bool is_mixed(const skel_ctx *c) {
  return c->prm.precision == SKEL_MIXED;
}

static int64_t to_doubles(bool f32, int64_t cnt) {
  return f32 ? (cnt + 1) / 2 : cnt;
}

static cudaError_t alloc_fac(skel_ctx *ctx, int64_t cnt, int64_t &off) {
  int64_t od = 0;
  cudaError_t e = ctx->fac.alloc(to_doubles(ctx->fac32, cnt), ctx->st, od);
  off = ctx->fac32 ? 2 * od : od;
  ctx->live_fac += to_doubles(ctx->fac32, cnt);
  return e;
}

static void fork_aux(skel_ctx *ctx) {
  cudaEventRecord(ctx->ev_fork, ctx->st);
  cudaStreamWaitEvent(ctx->st2, ctx->ev_fork, 0);
}

static void join_aux(skel_ctx *ctx) {
  cudaEventRecord(ctx->ev_join, ctx->st2);
  cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0);
}

// The boxes of one level by kernel: 0 one CTA each, 1 a 4-CTA cluster
// (mid-size boxes on levels of few boxes), 2 a 16-CTA cluster (large
// boxes).  The class depends only on the box and the tree.
struct LevelSel {
  std::vector<int32_t> h[3];  // positions in the level's LvlBox array
  const int32_t *d[3] = {nullptr, nullptr, nullptr};
  int max_n[3] = {0, 0, 0}, max_m[3] = {0, 0, 0};
  // the first `wide` boxes of class 2 are eliminated by whole-GPU launches
  // (k_wide.cu) instead of the cluster kernel; their sizes in wide_n
  int wide = 0, wide_qr = 0;  // the first wide_qr also take the wide CPQR
  std::vector<int> wide_n, wide_m;
  int n(int c) const { return (int)h[c].size(); }
};

// the streams (and their join events) of the wide boxes, created once
static cudaError_t wide_streams(skel_ctx *ctx, int nw) {
  cudaError_t ce = cudaSuccess;
  const int ns = std::min(nw, kWideStreams);
  for (int i = 0; i < ns && ce == cudaSuccess; ++i) {
    if (!ctx->wst[i]) {
      int lo = 0, hi = 0;
      cudaDeviceGetStreamPriorityRange(&lo, &hi);
      ce = cudaStreamCreateWithPriority(&ctx->wst[i], cudaStreamNonBlocking,
                                        hi);
    }
    if (ce == cudaSuccess && !ctx->wev[i])
      ce = cudaEventCreateWithFlags(&ctx->wev[i], cudaEventDisableTiming);
  }
  if (ce == cudaSuccess && !ctx->wev_fork)
    ce = cudaEventCreateWithFlags(&ctx->wev_fork, cudaEventDisableTiming);
  return ce;
}

// pinned stop flags and events for the host's reads during the wide CPQR
static cudaError_t qr_host_slots(skel_ctx *ctx, int nw) {
  if ((int)ctx->qr_events.size() < 2 * nw) {
    if (ctx->qr_hstop) cudaFreeHost((void *)ctx->qr_hstop);
    ctx->qr_hstop = nullptr;
    void *p = nullptr;
    cudaError_t ce = cudaMallocHost(&p, (size_t)2 * nw * sizeof(int32_t));
    if (ce != cudaSuccess) return ce;
    ctx->qr_hstop = static_cast<volatile int32_t *>(p);
    while ((int)ctx->qr_events.size() < 2 * nw) {
      cudaEvent_t e = nullptr;
      ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (ce != cudaSuccess) return ce;
      ctx->qr_events.push_back(e);
    }
  }
  return cudaSuccess;
}

// The kernels of one level: assembly, then CPQR and elimination with the
// one-CTA boxes on the main stream and the cluster boxes on the auxiliary
// one.  IdR: storage of the ID matrices; FacR: diagonal blocks and factors.
template <class IdR, class FacR>
static cudaError_t launch_level(skel_ctx *ctx, int level, int nb, int P,
                                const LevelSel &sel, int64_t tws_half) {
  IdR *dscr = reinterpret_cast<IdR *>(ctx->dscr.p);
  FacR *dsa = reinterpret_cast<FacR *>(ctx->dsa.p);
  FacR *fac = reinterpret_cast<FacR *>(ctx->fac.p);
  cudaError_t ce = cudaSuccess;
  static const int kCsOf[3] = {1, 4, 16};
  timed(ctx, KC_DIAG, [&] {
    launch_assemble_diag<FacR>(ctx->g, ctx->dlb.p, nb, ctx->iscr.p, dsa, fac,
                               ctx->st);
  });
  timed(ctx, KC_IDMAT, [&] {
    launch_assemble_id<IdR>(ctx->g, ctx->dlb.p, nb, ctx->iscr.p, dscr, P,
                            ctx->st);
  });
  timed(ctx, KC_CPQR, [&] {
    fork_aux(ctx);
    // the largest wide boxes (first of class 2) on the wide streams
    const int nw = sel.wide_qr;
    if (nw && ce == cudaSuccess) {
      std::vector<int> wq(sel.h[2].begin(), sel.h[2].begin() + nw);
      const std::vector<int> wn(sel.wide_n.begin(), sel.wide_n.begin() + nw);
      const std::vector<int> wm(sel.wide_m.begin(), sel.wide_m.begin() + nw);
      ce = wide_streams(ctx, nw);
      const int ns = std::min(nw, kWideStreams);
      const int mw = *std::max_element(wn.begin(), wn.end());
      if (ce == cudaSuccess)
        ce = ctx->qops.ensure((size_t)nw * qr_ops_bytes());
      if (ce == cudaSuccess) ce = ctx->qdws.ensure((size_t)nw * 2 * mw);
      if (ce == cudaSuccess) ce = ctx->qiws.ensure((size_t)nw * mw);
      if (ce == cudaSuccess) ce = ctx->qR.ensure((size_t)ns * mw * mw);
      if (ce == cudaSuccess) ce = qr_host_slots(ctx, nw);
      if (ce == cudaSuccess) {
        std::vector<cudaStream_t> sts(ctx->wst, ctx->wst + ns);
        cudaEventRecord(ctx->wev_fork, ctx->st2);
        for (cudaStream_t w : sts) cudaStreamWaitEvent(w, ctx->wev_fork, 0);
        ce = launch_cpqr_wide<IdR, FacR>(
            ctx->dlb.p, wq, wn, wm, ctx->iscr.p, dscr, ctx->dbox.p,
            fac, ctx->tws.p, ctx->prm.id_tol,
            reinterpret_cast<QrOps *>(ctx->qops.p), ctx->qdws.p,
            ctx->qiws.p, ctx->qR.p, sts, ctx->qr_hstop, ctx->qr_events);
        for (int i = 0; i < ns; ++i) {
          cudaEventRecord(ctx->wev[i], ctx->wst[i]);
          cudaStreamWaitEvent(ctx->st2, ctx->wev[i], 0);
        }
      }
    }
    for (int c = 2; c >= 1; --c) {
      const int off = c == 2 ? nw : 0;
      if (sel.n(c) > off && ce == cudaSuccess)
        ce = launch_cpqr_cluster<IdR, FacR>(
            ctx->dlb.p, sel.d[c] + off, sel.n(c) - off, ctx->iscr.p, dscr,
            ctx->dbox.p, fac, ctx->tws.p, ctx->prm.id_tol, sel.max_n[c],
            sel.max_m[c], ctx->st2, kCsOf[c]);
    }
    if (sel.n(0))
      launch_cpqr<IdR, FacR>(ctx->dlb.p, sel.d[0], sel.n(0), ctx->iscr.p, dscr,
                             ctx->dbox.p, fac, ctx->tws.p, ctx->prm.id_tol,
                             sel.max_n[0], ctx->st);
    join_aux(ctx);
  });
  if (ce != cudaSuccess) return ce;
  const int maxn = std::max(sel.max_n[0], std::max(sel.max_n[1],
                                                    sel.max_n[2]));
  // eliminate the boxes d[c][0..cnt[c]) of each class; the first of class
  // 2 (wq: their positions, wn: their sizes) by whole-GPU launches
  auto eliminate = [&](const int32_t *const d[3], const int cnt[3],
                       const std::vector<int> &wq, const std::vector<int> &wn,
                       int allow_move) {
    timed(ctx, KC_ELIM, [&] {
      fork_aux(ctx);
      const int nw = (int)wq.size();
      if (nw && ce == cudaSuccess) {
        if constexpr (std::is_same<FacR, double>::value) {
          const int mw = *std::max_element(wn.begin(), wn.end());
          const int ns = std::min(nw, kWideStreams);
          ce = wide_streams(ctx, nw);
          if (ce == cudaSuccess) ce = ctx->wkp.ensure((size_t)ns * mw * mw);
          // the first pass keeps X_RR of every box for a possible split,
          // and its descriptors live until then (the second pass, over
          // the flagged boxes only, runs after the split)
          if (ce == cudaSuccess && allow_move)
            ce = ctx->wxs.ensure((size_t)nw * mw * mw);
          if (ce == cudaSuccess)
            ce = ctx->wiws.ensure((size_t)nw * 2 * mw);
          if (ce == cudaSuccess)
            ce = ctx->wops.ensure((size_t)nw * wide_ops_bytes());
          if (ce == cudaSuccess) {
            // the wide streams start after st2's pending work and st2
            // continues after all of them
            std::vector<cudaStream_t> sts(ctx->wst, ctx->wst + ns);
            cudaEventRecord(ctx->wev_fork, ctx->st2);
            for (cudaStream_t w : sts) cudaStreamWaitEvent(w, ctx->wev_fork, 0);
            ce = launch_eliminate_wide(
                ctx->dlb.p, wq, wn, ctx->iscr.p, dsa, ctx->dbox.p, fac,
                ctx->ipool.p, ctx->dofs.p, ctx->wkp.p, ctx->wxs.p,
                ctx->wiws.p, reinterpret_cast<WideOps *>(ctx->wops.p),
                ctx->dstatus.p, allow_move, ctx->dflag.p,
                is_mixed(ctx) && ctx->tc_products, sts);
            for (int i = 0; i < ns; ++i) {
              cudaEventRecord(ctx->wev[i], ctx->wst[i]);
              cudaStreamWaitEvent(ctx->st2, ctx->wev[i], 0);
            }
          }
        }
      }
      for (int c = 2; c >= 1; --c) {
        const int off = c == 2 ? nw : 0;
        if (cnt[c] > off && ce == cudaSuccess)
          ce = launch_eliminate_cluster<FacR>(
              ctx->dlb.p, d[c] + off, cnt[c] - off, ctx->iscr.p, dsa,
              ctx->dbox.p, fac, ctx->ipool.p, ctx->dofs.p, sel.max_n[c],
              ctx->dstatus.p, allow_move, ctx->dflag.p, ctx->st2, kCsOf[c]);
      }
      if (cnt[0])
        launch_eliminate<FacR>(ctx->dlb.p, d[0], cnt[0], ctx->iscr.p, dsa,
                               ctx->dbox.p, fac, ctx->ipool.p, ctx->dofs.p,
                               sel.max_n[0], ctx->dstatus.p, allow_move,
                               ctx->dflag.p, ctx->st);
      join_aux(ctx);
    });
  };
  {
    const int cnt[3] = {sel.n(0), sel.n(1), sel.n(2)};
    const std::vector<int> wq(sel.h[2].begin(), sel.h[2].begin() + sel.wide);
    eliminate(sel.d, cnt, wq, sel.wide_n, 1);
  }
  if (ce != cudaSuccess) return ce;
  // X_RR conditioning (Sec. 2.2 remark): boxes whose X_RR LU was flagged
  // move the indices found by the diagonal-pivoting split from R into S and
  // are eliminated again (the second time without flagging; a still
  // singular X_RR is then reported by the 1e-14 pivot test).
  std::vector<int32_t> hflag(nb), hmoves(nb);
  if ((ce = sync_st(ctx)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(hflag.data(), ctx->dflag.p, nb * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, ctx->st)) != cudaSuccess ||
      (ce = sync_st(ctx)) != cudaSuccess)
    return ce;
  // [flagged, class by class | the same again | moved]
  std::vector<int32_t> lists;
  int fcnt[3] = {0, 0, 0};
  std::vector<int> fwq, fwn, fwb;  // flagged wide boxes (first in class 2)
  std::vector<int32_t> nonwide;      // the other flagged boxes
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < sel.n(c); ++i) {
      const int32_t q = sel.h[c][i];
      if (!hflag[q]) continue;
      lists.push_back(q);
      ++fcnt[c];
      if (c == 2 && i < sel.wide) {
        fwq.push_back(q);
        fwn.push_back(sel.wide_n[i]);
        fwb.push_back(i);  // its descriptor in the first pass
      } else {
        nonwide.push_back(q);
      }
    }
  const int nf = (int)lists.size();
  if (nf == 0) return cudaSuccess;
  const std::vector<int32_t> flagged(lists.begin(), lists.end());
  lists.insert(lists.end(), flagged.begin(), flagged.end());
  // [flagged | flagged | moved (<= nf) | flagged, not wide]
  if ((ce = ctx->dfsel.ensure(4 * nf + 1)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(ctx->dfsel.p, lists.data(),
                            lists.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, ctx->st)) != cudaSuccess)
    return ce;
  if (!nonwide.empty() &&
      (ce = cudaMemcpyAsync(ctx->dfsel.p + 3 * nf, nonwide.data(),
                            nonwide.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, ctx->st)) != cudaSuccess)
    return ce;
  const int32_t *dfall = ctx->dfsel.p;
  const int32_t *dfc[3] = {dfall + nf, dfall + nf + fcnt[0],
                           dfall + nf + fcnt[0] + fcnt[1]};
  timed(ctx, KC_ELIM, [&] {
    // the flagged wide boxes split their saved X_RR with whole-GPU
    // launches, the others on a cluster each
    // one flagged wide box per wide stream (forked from st, joined after
    // the cluster splits on st have been enqueued beside them)
    int forked = 0;
    if (!fwq.empty()) {
      if constexpr (std::is_same<FacR, double>::value) {
        const int nw = (int)fwq.size();
        const int ns = std::min(nw, kWideStreams);
        ce = wide_streams(ctx, nw);
        if (ce == cudaSuccess) {
          std::vector<cudaStream_t> sts(ctx->wst, ctx->wst + ns);
          cudaEventRecord(ctx->wev_fork, ctx->st);
          for (cudaStream_t w : sts) cudaStreamWaitEvent(w, ctx->wev_fork, 0);
          forked = ns;
          ce = launch_xrr_split_wide(ctx->dlb.p, fwq, fwn, fwb, ctx->dbox.p,
                                     ctx->ipool.p,
                                     reinterpret_cast<WideOps *>(ctx->wops.p),
                                     ctx->dmoves.p, sts);
        }
      }
    }
    if (ce == cudaSuccess && !nonwide.empty())
      ce = launch_xrr_split_cluster<FacR>(
          ctx->dlb.p, dfall + 3 * nf, (int)nonwide.size(), ctx->iscr.p, dsa,
          ctx->dbox.p, fac, ctx->ipool.p, ctx->dmoves.p, maxn, ctx->st);
    for (int i = 0; i < forked; ++i) {
      cudaEventRecord(ctx->wev[i], ctx->wst[i]);
      cudaStreamWaitEvent(ctx->st, ctx->wev[i], 0);
    }
  });
  if (ce != cudaSuccess) return ce;
  if ((ce = sync_st(ctx)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(hmoves.data(), ctx->dmoves.p,
                            nb * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->st)) != cudaSuccess ||
      (ce = sync_st(ctx)) != cudaSuccess)
    return ce;
  std::vector<int32_t> mv;
  for (int t = 0; t < nf; ++t)
    if (hmoves[lists[t]] > 0) {
      mv.push_back(lists[t]);
      ctx->lv_moved[level] += hmoves[lists[t]];
    }
  if (!mv.empty()) {
    if ((ce = cudaMemcpyAsync(ctx->dfsel.p + 2 * nf, mv.data(),
                              mv.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, ctx->st)) != cudaSuccess)
      return ce;
    timed(ctx, KC_ELIM, [&] {
      launch_repartition<FacR>(ctx->dlb.p, ctx->dfsel.p + 2 * nf,
                               (int)mv.size(), ctx->iscr.p, ctx->dbox.p, fac,
                               ctx->ipool.p, ctx->dmoves.p, ctx->tws.p,
                               tws_half, maxn, ctx->st);
    });
  }
  eliminate(dfc, fcnt, fwq, fwn, 0);
  return ce;
}

// level sweeps with the factors in their storage type
static void sweep_up_jobs(skel_ctx *ctx, int l, const UpJobs &jobs, int njobs,
                          int64_t ld, int nrhs) {
  const int nb = (int)ctx->tree.levels[l].size();
  const int32_t *ids = ctx->lvl_ids.p + ctx->lvl_off[l];
  if (ctx->fac32)
    launch_up_sweep<float>(ctx->dbox.p, ids, nb, ctx->dofs.p,
                           reinterpret_cast<const float *>(ctx->fac.p),
                           ctx->ipool.p, jobs, njobs, ld, nrhs,
                           ctx->lv_alln[l], ctx->sweep_rhs_chunk,
                           ctx->dstatus.p, ctx->st);
  else
    launch_up_sweep<double>(ctx->dbox.p, ids, nb, ctx->dofs.p, ctx->fac.p,
                            ctx->ipool.p, jobs, njobs, ld, nrhs,
                            ctx->lv_alln[l], ctx->sweep_rhs_chunk,
                            ctx->dstatus.p, ctx->st);
}

static void sweep_up(skel_ctx *ctx, int l, double *b, int64_t ld, int nrhs,
                     double *pre, int mode) {
  // no initial columns (b holds the input) and no snapshots
  UpJobs j{{b, nullptr}, {pre, nullptr}, {mode, 0}, {nullptr, nullptr},
           nullptr};
  sweep_up_jobs(ctx, l, j, 1, ld, nrhs);
}

static void sweep_down(skel_ctx *ctx, int l, double *x, int64_t ld, int nrhs,
                       int mode) {
  const int nb = (int)ctx->tree.levels[l].size();
  const int32_t *ids = ctx->lvl_ids.p + ctx->lvl_off[l];
  if (ctx->fac32)
    launch_down_sweep<float>(ctx->dbox.p, ids, nb, ctx->dofs.p,
                             reinterpret_cast<const float *>(ctx->fac.p), x,
                             ld, nrhs, mode, ctx->lv_alln[l],
                             ctx->sweep_rhs_chunk, ctx->dstatus.p, ctx->st);
  else
    launch_down_sweep<double>(ctx->dbox.p, ids, nb, ctx->dofs.p, ctx->fac.p,
                              x, ld, nrhs, mode, ctx->lv_alln[l],
                              ctx->sweep_rhs_chunk, ctx->dstatus.p, ctx->st);
}

// ---------------------------------------------------------------------------
// one level of compression over the boxes in `work` (ids at depth `level`)

static int compress_level(skel_ctx *ctx, int level,
                          const std::vector<int> &work) {
  const Tree &t = ctx->tree;
  const int P = ctx->prm.n_proxy;
  const double ratio = ctx->prm.proxy_ratio;
  const int nb = (int)work.size();
  if (nb == 0) return SKEL_OK;
  ctx->cur_level = level;
  struct LevelTag {
    skel_ctx *c;
    ~LevelTag() { c->cur_level = 0; }
  } level_tag{ctx};
  const double tp0 = now_ms();
  std::vector<LvlBox> lb(nb);
  std::vector<int32_t> ibuf;
  int64_t dtot = 0, atot = 0, ttot = 0;
  int max_n = 0, max_m = 0;
  std::vector<int32_t> act, fint;
  std::vector<int> near;
  for (int q = 0; q < nb; ++q) {
    const int b = work[q];
    const HBox &B = t.boxes[b];
    level_act(ctx, b, act);
    near_owners(t, b, level, ratio, near);
    ctx->hnear[b] = near;
    const double rho = proxy_radius(B, ratio);
    // the near owners' active DOFs inside the proxy disk, in the order of
    // their active lists (children's skeletons, or a leaf's nodes)
    fint.clear();
    const double rr = rho * rho;
    auto inside = [&](int64_t j) {
      const double ex = ctx->hx[j] - B.cx, ey = ctx->hy[j] - B.cy;
      return ex * ex + ey * ey < rr;
    };
    for (int o : near) {
      const HBox &O = t.boxes[o];
      if (!O.leaf) {  // an owner of this level: its children's skeletons
        for (int c = 0; c < O.nchild; ++c) {
          const int cb = O.child[c];
          const int32_t *d = ctx->hdofs[cb].data();
          for (int i = 0, k = ctx->hbox[cb].k; i < k; ++i)
            if (inside(dof_node(ctx, d[i]))) fint.push_back(d[i]);
        }
      } else {  // a leaf (of this level or above): its nodes' DOFs
        for (int64_t i = O.nbeg; i < O.nbeg + O.ncnt; ++i) {
          const int64_t j = ctx->tree.order[i];
          if (!inside(j)) continue;
          if (ctx->dpn == 1) {
            fint.push_back((int32_t)j);
          } else {
            fint.push_back((int32_t)(2 * j));
            fint.push_back((int32_t)(2 * j + 1));
          }
        }
      }
    }
    LvlBox &L = lb[q];
    L.box = b;
    L.n = (int)act.size();
    L.nf = (int)fint.size();
    L.m = 2 * L.nf + (ctx->lap ? 4 : 6) * P + 2;
    L.nchild = B.leaf ? 0 : B.nchild;
    int seg = 0;
    for (int c = 0; c < 4; ++c) {
      L.cseg[c] = 0;
      L.ck[c] = 0;
      L.cxss[c] = 0;
    }
    for (int c = 0; c < L.nchild; ++c) {
      const DevBox &C = ctx->hbox[B.child[c]];
      L.cseg[c] = seg;
      L.ck[c] = C.k;
      L.cxss[c] = C.fac_off + fac_XSS(C.k, C.n - C.k);
      seg += C.k;
    }
    L.act_off = (int64_t)ibuf.size();
    ibuf.insert(ibuf.end(), act.begin(), act.end());
    L.fint_off = (int64_t)ibuf.size();
    ibuf.insert(ibuf.end(), fint.begin(), fint.end());
    L.perm_off = (int64_t)ibuf.size();
    ibuf.resize(ibuf.size() + L.n);
    while (ibuf.size() % 8) ibuf.push_back(0);
    L.a_off = atot;
    atot += ((int64_t)L.n * L.n + 31) / 32 * 32;
    L.m_off = dtot;
    dtot += ((int64_t)L.m * L.n + 31) / 32 * 32;
    L.t_off = ttot;
    ttot += ((int64_t)L.n * L.n / 4 + 1 + 31) / 32 * 32;
    L.cx = B.cx;
    L.cy = B.cy;
    L.rho = rho;
    max_n = std::max(max_n, L.n);
    max_m = std::max(max_m, L.m);
    DevBox &D = ctx->hbox[b];
    D.n = L.n;
    D.k = 0;
    D.leaf = B.leaf ? 1 : 0;
    D.snap_off = -1;  // assigned once the rank is known (factor_all)
    // an arena that grows moves: the sweeps on st3 read it
    if (!ctx->fac.fits(to_doubles(ctx->fac32, fac_region(L.n))) ||
        !ctx->ipool.fits(std::max(L.n, 1)) || !ctx->dofs.fits(std::max(L.n, 1)))
      CU(cudaStreamSynchronize(ctx->st3));
    CU(alloc_fac(ctx, fac_region(L.n), D.fac_off));
    CU(ctx->ipool.alloc(std::max(L.n, 1), ctx->st, D.piv_off));
    CU(ctx->dofs.alloc(std::max(L.n, 1), ctx->st, D.dof_off));
  }
  if (max_n > 12000)
    return fail(ctx, SKEL_ECAPACITY,
                "box with " + std::to_string(max_n) + " active DOFs");
  // Large boxes go to the cluster kernels (many SMs per box); every box of
  // a level with few boxes counts as large once it has more active DOFs
  // than a full leaf.  The choice depends only on the box and the tree (not
  // on how many boxes are being recompressed), so an update and a fresh
  // factorization run every box through the same kernel and agree bit for
  // bit.
  const int level_boxes = (int)t.levels[level].size();
  LevelSel sel;
  for (int q = 0; q < nb; ++q) {
    const int n = lb[q].n;
    const bool big = n >= ctx->cluster_min_n ||
                     (level_boxes <= ctx->cluster_level_boxes &&
                      n > 2 * ctx->prm.leaf_size);
    const bool mid = !big && level_boxes <= ctx->cluster_mid_level_boxes &&
                     n >= ctx->cluster_mid_min_n;
    const int c = big ? 2 : mid ? 1 : 0;
    sel.h[c].push_back(q);
    sel.max_n[c] = std::max(sel.max_n[c], n);
    sel.max_m[c] = std::max(sel.max_m[c], lb[q].m);
  }
  // largest boxes first (work about m n^2 for the CPQR and n^3 for the
  // elimination): the CTAs of a launch start in index order, so the long
  // ones no longer trail at the end while other SMs idle.  Each box's
  // result does not depend on the order.
  for (int c = 0; c < 3; ++c)
    std::stable_sort(sel.h[c].begin(), sel.h[c].end(), [&](int a, int b) {
      const double wa = (double)lb[a].m * lb[a].n * lb[a].n;
      const double wb = (double)lb[b].m * lb[b].n * lb[b].n;
      return wa > wb;
    });
  // the largest boxes of class 2 are eliminated by whole-GPU launches
  // (FP64 factors only); they go first in the class, largest first
  if (!ctx->fac32) {
    auto is_wide = [&](int q) { return lb[q].n >= ctx->wide_min_n; };
    std::stable_partition(sel.h[2].begin(), sel.h[2].end(), is_wide);
    for (int q : sel.h[2]) {
      if (!is_wide(q)) break;
      ++sel.wide;
    }
    // Of those, the largest also take the whole-GPU CPQR (first), when the
    // level of the tree has at least two such boxes: its per-step latency
    // is hidden only by several boxes on their streams at once (a single
    // 2548-DOF box: 77 ms against 62 on its cluster; four to sixteen
    // boxes of 1700-3300 DOFs: 1.5-2x faster).  The count runs over every
    // box of the level, the ones not recompressed by an update with their
    // kept sizes, so updates and fresh factorizations route alike.
    int level_wqr = 0;
    {
      std::unordered_map<int, int> nwork;
      for (int q = 0; q < nb; ++q) nwork[work[q]] = lb[q].n;
      for (int b : t.levels[level]) {
        auto it = nwork.find(b);
        const int nb_ = it != nwork.end() ? it->second : ctx->hbox[b].n;
        if (nb_ >= ctx->wide_qr_min_n) ++level_wqr;
      }
    }
    auto is_wqr = [&](int q) {
      return level_wqr >= 2 && lb[q].n >= ctx->wide_qr_min_n;
    };
    std::stable_partition(sel.h[2].begin(), sel.h[2].begin() + sel.wide,
                          is_wqr);
    for (int i = 0; i < sel.wide; ++i) {
      const int q = sel.h[2][i];
      sel.wide_n.push_back(lb[q].n);
      sel.wide_m.push_back(lb[q].m);
      if (is_wqr(q)) ++sel.wide_qr;
    }
  }
  int64_t sel_off[3];
  for (int c = 0; c < 3; ++c) {
    sel_off[c] = (int64_t)ibuf.size();
    ibuf.insert(ibuf.end(), sel.h[c].begin(), sel.h[c].end());
  }
  CU(ctx->dlb.ensure(nb));
  CU(ctx->iscr.ensure(ibuf.size() + 1));
  CU(ctx->dscr.ensure(to_doubles(ctx->id32, dtot) + 1));
  CU(ctx->dsa.ensure(to_doubles(ctx->fac32, atot) + 1));
  CU(ctx->tws.ensure(2 * ttot + 1));  // second half: repartition scratch
  CU(ctx->dbox.ensure(ctx->hbox.size()));
  CU(cudaMemcpyAsync(ctx->dlb.p, lb.data(), nb * sizeof(LvlBox),
                     cudaMemcpyHostToDevice, ctx->st));
  CU(cudaMemcpyAsync(ctx->iscr.p, ibuf.data(), ibuf.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, ctx->st));
  CU(cudaMemcpyAsync(ctx->dbox.p, ctx->hbox.data(),
                     ctx->hbox.size() * sizeof(DevBox), cudaMemcpyHostToDevice,
                     ctx->st));
  ctx->host_prep_ms += now_ms() - tp0;
  CU(cudaMemsetAsync(ctx->dstatus.p, 0, sizeof(int), ctx->st));
  for (int c = 0; c < 3; ++c) sel.d[c] = ctx->iscr.p + sel_off[c];
  cudaError_t lce;
  CU(ctx->dflag.ensure(nb));
  CU(ctx->dmoves.ensure(nb));
  CU(cudaMemsetAsync(ctx->dmoves.p, 0, nb * sizeof(int32_t), ctx->st));
  if (ctx->fac32)
    lce = launch_level<float, float>(ctx, level, nb, P, sel, ttot);
  else if (ctx->id32)
    lce = launch_level<float, double>(ctx, level, nb, P, sel, ttot);
  else
    lce = launch_level<double, double>(ctx, level, nb, P, sel, ttot);
  CU(lce);
  ctx->lv_big[level] = sel.n(2) + sel.n(1);
  ctx->lv_wide[level] = sel.wide;
  CU(cudaGetLastError());
  // read back ranks and the permuted active lists (the parents need them)
  CU(sync_st(ctx));  // (a copy into pageable memory waits as well)
  CU(cudaMemcpyAsync(ctx->hbox.data(), ctx->dbox.p,
                     ctx->hbox.size() * sizeof(DevBox), cudaMemcpyDeviceToHost,
                     ctx->st));
  int status = 0;
  CU(cudaMemcpyAsync(&status, ctx->dstatus.p, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->st));
  CU(sync_st(ctx));
  const double tq0 = now_ms();
  // one copy of the level's slice of the DOF arena (the boxes' lists were
  // allocated one after another), then split on the host
  int64_t lo = INT64_MAX, hi = 0;
  for (int q = 0; q < nb; ++q) {
    const DevBox &D = ctx->hbox[work[q]];
    lo = std::min(lo, D.dof_off);
    hi = std::max(hi, D.dof_off + std::max(D.n, 1));
  }
  std::vector<int32_t> slice(hi > lo ? hi - lo : 0);
  if (!slice.empty()) {
    CU(cudaMemcpyAsync(slice.data(), ctx->dofs.p + lo,
                       slice.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->st));
    CU(sync_st(ctx));
  }
  for (int q = 0; q < nb; ++q) {
    const DevBox &D = ctx->hbox[work[q]];
    auto &v = ctx->hdofs[work[q]];
    v.assign(slice.begin() + (D.dof_off - lo),
             slice.begin() + (D.dof_off - lo) + D.n);
  }
  resolve_timing(ctx);
  if (status == SKEL_ESINGULAR)
    return fail(ctx, SKEL_ESINGULAR,
                "X_RR pivot ratio below 1e-14 at level " +
                    std::to_string(level));
  if (status != 0)
    return fail(ctx, status,
                "a compression kernel reported an error at level " +
                    std::to_string(level));
  // statistics: algorithmic work of every box from its realised sizes
  int mk = 0;
  for (int q = 0; q < nb; ++q) {
    const DevBox &D = ctx->hbox[work[q]];
    const LvlBox &L = lb[q];
    mk = std::max(mk, D.k);
    const double n = D.n, k = D.k, r = D.n - D.k, m = L.m;
    // Householder steps j < k on the trailing (m-j) x (n-j-1) block, then
    // the triangular solve for T
    double qr = 0.0;
    for (int j = 0; j < D.k; ++j) qr += 4.0 * (m - j) * (n - j - 1);
    qr += k * k * r;
    const double el = 2 * r * k * k + 2 * k * k * r + 4 * k * r * r +
                      2.0 * r * r * r / 3.0 + 4 * r * r * k + 2 * k * k * r;
    ctx->kst[KC_CPQR].flops += qr;
    ctx->kst[KC_CPQR].bytes += 8.0 * m * n;
    ctx->kst[KC_ELIM].flops += el;
    ctx->kst[KC_ELIM].bytes += 8.0 * (n * n + n * n + k * r);
    ctx->kst[KC_IDMAT].flops += kEntryFlops * m * n;
    ctx->kst[KC_IDMAT].bytes += 8.0 * m * n;
    ctx->kst[KC_DIAG].flops += kEntryFlops * n * n;
    ctx->kst[KC_DIAG].bytes += 8.0 * n * n;
    ctx->flops_factor += qr + el + kEntryFlops * (m * n + n * n);
  }
  ctx->host_post_ms += now_ms() - tq0;
  ctx->lv_nbox[level] = nb;
  ctx->lv_maxn[level] = max_n;
  ctx->lv_maxk[level] = mk;
  ctx->lv_maxm[level] = max_m;
  return SKEL_OK;
}

// Root block, bordering columns and the top dense LU (Sec. 3.2).
static int factor_top(skel_ctx *ctx) {
  const Tree &t = ctx->tree;
  const HBox &R = t.boxes[0];
  const int64_t n2 = ndof(ctx);
  const int p3 = nbord(ctx);
  level_act(ctx, 0, ctx->root_act);
  ctx->s = (int)ctx->root_act.size();
  const int s = ctx->s;
  ctx->ldt = s + p3;
  const int ldt = ctx->ldt;
  LvlBox L{};
  L.box = 0;
  L.n = s;
  L.nchild = R.leaf ? 0 : R.nchild;
  int seg = 0;
  for (int c = 0; c < L.nchild; ++c) {
    const DevBox &C = ctx->hbox[R.child[c]];
    L.cseg[c] = seg;
    L.ck[c] = C.k;
    L.cxss[c] = C.fac_off + fac_XSS(C.k, C.n - C.k);
    seg += C.k;
  }
  L.act_off = 0;
  CU(ctx->dlb.ensure(1));
  CU(ctx->iscr.ensure(s + 1));
  CU(ctx->droot_act.ensure(s + 1));
  CU(cudaMemcpyAsync(ctx->dlb.p, &L, sizeof L, cudaMemcpyHostToDevice,
                     ctx->st));
  CU(cudaMemcpyAsync(ctx->iscr.p, ctx->root_act.data(), s * sizeof(int32_t),
                     cudaMemcpyHostToDevice, ctx->st));
  CU(cudaMemcpyAsync(ctx->droot_act.p, ctx->root_act.data(),
                     s * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
  // + the LU's pivot statistics, panel row map and reciprocal pivots
  CU(ctx->top.ensure((size_t)ldt * ldt + lu_extra_doubles(ldt)));
  CU(ctx->top_piv.ensure(ldt + 1));
  timed(ctx, KC_DIAG, [&] {
    if (ctx->fac32)
      launch_root_block<float>(ctx->g, ctx->dlb.p, ctx->iscr.p,
                               reinterpret_cast<const float *>(ctx->fac.p),
                               ctx->top.p, ldt, ctx->st);
    else
      launch_root_block<double>(ctx->g, ctx->dlb.p, ctx->iscr.p, ctx->fac.p,
                                ctx->top.p, ldt, ctx->st);
  });
  // rmask: every DOF eliminated below the root
  std::vector<uint8_t> mask(n2, 1);
  for (int32_t d : ctx->root_act) mask[d] = 0;
  CU(ctx->rmask.ensure(n2));
  CU(cudaMemcpyAsync(ctx->rmask.p, mask.data(), n2, cudaMemcpyHostToDevice,
                     ctx->st));
  CU(cudaMemsetAsync(ctx->dstatus.p, 0, sizeof(int), ctx->st));
  if (p3 > 0) {
    const size_t sz = (size_t)n2 * p3;
    CU(ctx->UH.ensure(sz));
    CU(ctx->W.ensure(sz));
    CU(ctx->QT.ensure(sz));
    CU(ctx->Wt.ensure(sz));
    CU(ctx->G.ensure((size_t)p3 * p3));
    CU(ctx->gscr_i.ensure(gram_scratch_ints(n2, p3)));
    if (ctx->bs.on) {
      // the level sweeps (bord_level) are done on st3
      CU(cudaEventRecord(ctx->ev_join3, ctx->st3));
      CU(cudaStreamWaitEvent(ctx->st, ctx->ev_join3, 0));
    } else {  // the root is a leaf: the top block takes H and Psi as they are
      timed(ctx, KC_BORDER, [&] {
        launch_h_columns(ctx->g, ctx->W.p, n2, ctx->st);
        launch_psi_columns(ctx->g, ctx->Wt.p, n2, ctx->st);
      });
    }
    timed(ctx, KC_GRAM, [&] {
      launch_gram_masked(ctx->QT.p, ctx->W.p, n2, n2, p3, ctx->rmask.p,
                         ctx->gscr_i.p, ctx->G.p, ctx->st);
      launch_top_fill(ctx->top.p, ldt, s, p3, ctx->droot_act.p, ctx->W.p,
                      ctx->Wt.p, n2, ctx->G.p, ctx->st);
    });
    ctx->kst[KC_GRAM].flops += 2.0 * n2 * p3 * p3;
    ctx->kst[KC_GRAM].bytes += 16.0 * n2 * p3;
  }
  int dummy = 0;
  timed(ctx, KC_TOPLU, [&] {
    launch_dense_lu(ctx->top.p, ldt, ldt, ctx->top_piv.p, &dummy, ctx->st);
  });
  ctx->kst[KC_TOPLU].flops += 2.0 / 3.0 * (double)ldt * ldt * ldt;
  ctx->kst[KC_TOPLU].bytes += 8.0 * (double)ldt * ldt;
  CU(cudaGetLastError());
  double ustat[2] = {0, 0};
  int status = 0;
  CU(sync_st(ctx));
  CU(cudaMemcpyAsync(ustat, ctx->top.p + (size_t)ldt * ldt, 2 * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->st));
  CU(cudaMemcpyAsync(&status, ctx->dstatus.p, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->st));
  int status3 = 0;
  if (ctx->bs.on)
    CU(cudaMemcpyAsync(&status3, ctx->dstatus3.p, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->st));
  CU(sync_st(ctx));
  resolve_timing(ctx);
  resolve_timing3(ctx);  // st waited for st3 above
  if (status3 != 0) status = status3;
  if (status != 0)
    return fail(ctx, status, "a bordered sweep kernel rejected a box");
  if (ldt > 0 && !(ustat[1] > 1e-15 * ustat[0]))
    return fail(ctx, SKEL_ESINGULAR, "top block is numerically singular");
  ctx->flops_factor += 2.0 / 3.0 * (double)ldt * ldt * ldt;
  return SKEL_OK;
}

static int upload_level_ids(skel_ctx *ctx) {
  const Tree &t = ctx->tree;
  std::vector<int32_t> ids;
  ctx->lvl_off.assign(t.levels.size() + 1, 0);
  for (size_t l = 0; l < t.levels.size(); ++l) {
    ctx->lvl_off[l] = (int64_t)ids.size();
    ids.insert(ids.end(), t.levels[l].begin(), t.levels[l].end());
  }
  CU(ctx->lvl_ids.ensure(ids.size() + 1));
  CU(cudaMemcpyAsync(ctx->lvl_ids.p, ids.data(), ids.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, ctx->st));
  return SKEL_OK;
}

static void reset_stats(skel_ctx *ctx) {
  const size_t nl = ctx->tree.levels.size();
  ctx->lv_nbox.assign(nl, 0);
  ctx->lv_maxn.assign(nl, 0);
  ctx->lv_maxk.assign(nl, 0);
  ctx->lv_maxm.assign(nl, 0);
  ctx->lv_big.assign(nl, 0);
  ctx->lv_wide.assign(nl, 0);
  ctx->lv_kms.assign(nl, std::vector<double>(KC_N, 0.0));
  ctx->lv_moved.assign(nl, 0);
  ctx->lv_ms.assign(nl, 0.0);
  ctx->flops_factor = 0;
}

// A region of the pinned staging buffer for an upload on st3.  When it
// must grow, st3 is drained first (the copies from the old one are done).
static void *pin_take(skel_ctx *ctx, size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  if (ctx->pin_used + bytes > ctx->pin_cap) {
    cudaStreamSynchronize(ctx->st3);
    const size_t nc = std::max({2 * ctx->pin_cap, bytes, (size_t)1 << 20});
    if (ctx->pin) cudaFreeHost(ctx->pin);
    ctx->pin = nullptr;
    ctx->pin_cap = ctx->pin_used = 0;
    if (cudaMallocHost(&ctx->pin, nc) != cudaSuccess) return nullptr;
    ctx->pin_cap = nc;
  }
  void *p = ctx->pin + ctx->pin_used;
  ctx->pin_used += bytes;
  return p;
}

// Start of the bordered sweeps (Sec. 3.2) of one factorization: buffers,
// and H and Psi on the sweep stream st3 once the geometry is there.
static int bord_begin(skel_ctx *ctx, const std::vector<char> *dirty) {
  BordState &S = ctx->bs;
  const Tree &t = ctx->tree;
  S = BordState{};
  const int p3 = nbord(ctx);
  const int64_t n2 = ndof(ctx);
  if (p3 == 0 || t.boxes[0].leaf || t.L() < 1) return SKEL_OK;
  S.on = true;
  S.full_b = !dirty || ctx->bord_full;
  S.dirty = S.full_b ? nullptr : dirty;
  CU(cudaStreamSynchronize(ctx->st3));  // buffers below may move
  ctx->pin_used = 0;
  const size_t sz = (size_t)n2 * p3;
  CU(ctx->UH.ensure(sz));
  CU(ctx->W.ensure(sz));
  CU(ctx->QT.ensure(sz));
  CU(ctx->Wt.ensure(sz));
  CU(ctx->H0.ensure(sz));
  CU(ctx->P0.ensure(sz));
  if (S.full_b) ctx->snap.used = 0;
  // items (box, chunk, job) of every level, at most boxes x 3p x 2, and up
  // to four restores per item, 3 ints each
  CU(ctx->sitems.ensure((size_t)t.boxes.size() * p3 * 2 * 3 * 5 + 1));
  CU(ctx->dbox_sw.ensure(ctx->hbox.size()));
  CU(ctx->dstatus3.ensure(1));
  S.lv_q.assign(t.L() + 2, 0);
  S.col_prev.assign(p3, 0);
  for (int a = 0; a < p3 && a < (int)ctx->bord_col_changed.size(); ++a)
    S.col_prev[a] = ctx->bord_col_changed[a];
  // the geometry (and an update's renumbered DOF lists) arrive on st
  CU(cudaEventRecord(ctx->ev_fork3, ctx->st));
  CU(cudaStreamWaitEvent(ctx->st3, ctx->ev_fork3, 0));
  CU(cudaMemsetAsync(ctx->dstatus3.p, 0, sizeof(int), ctx->st3));
  timed_on(ctx, KC_BORDER, ctx->st3, [&] {
    launch_h_columns(ctx->g, ctx->H0.p, n2, ctx->st3);
    launch_psi_columns(ctx->g, ctx->P0.p, n2, ctx->st3);
  });
  return SKEL_OK;
}

// The bordered sweeps of level l, once its factors exist (the host holds
// its boxes' records).  Work items (box, chunk, job), job 0 = U on H, 1 =
// V^T on Psi.  After an update only some are swept again: column a of job
// j for box b when b was recompressed, or (H only) when a lies in the
// level's set of swept columns: the level's chunks that meet a changed
// column (the H columns of a hole whose centre moved change at every node)
// or a column swept on the level below.  A box thus sweeps every column
// any of its children sweeps, and its rows in W are rewritten after
// theirs; columns swept without a change have unchanged inputs and give
// unchanged outputs.  A swept box reads its children's b_S rows, which its
// own last sweep overwrote, so the children that did not sweep all of its
// chunk restore them from their snapshots first.  If the level's chunk
// width differs from the last sweep's, this level and those above are
// swept completely (the kept outputs were made with the old chunking).
static int bord_level(skel_ctx *ctx, int l) {
  BordState &S = ctx->bs;
  if (!S.on) return SKEL_OK;
  const Tree &t = ctx->tree;
  const int p3 = nbord(ctx);
  const int64_t n2 = ndof(ctx);
  const auto &lb = t.levels[l];
  const std::vector<char> *dirty = S.dirty;
  for (int b : lb)
    if (S.full_b || (*dirty)[b]) {
      DevBox &D = ctx->hbox[b];
      // (a growing arena is copied on st3, after the sweeps that use it)
      CU(ctx->snap.alloc(std::max<int64_t>(2 * (int64_t)D.k * p3, 1),
                         ctx->st3, D.snap_off));
    }
  int maxn = 0;
  for (int b : lb) maxn = std::max(maxn, ctx->hbox[b].n);
  const int q = sweep_chunk((int)lb.size(), 2, p3, maxn, ctx->sweep_rhs_chunk);
  S.lv_q[l] = q;
  if ((int)ctx->bord_lv_q.size() != t.L() + 2 || ctx->bord_lv_q[l] != q)
    S.full = true;
  const bool all = !dirty || S.full;
  std::vector<char> col(p3, 0);
  for (int c = 0; c * q < p3; ++c) {
    bool any = false;
    for (int a = c * q; a < std::min(p3, (c + 1) * q); ++a)
      any = any || S.col_prev[a];
    for (int a = c * q; a < std::min(p3, (c + 1) * q); ++a) col[a] = any;
  }
  auto swept = [&](int b, int c, int job) {
    return all || (*dirty)[b] || (job == 0 && col[c * q]);
  };
  // a child (level l + 1) swept every column of [a0, a1)
  auto child_swept = [&](int b, int a0, int a1, int job) {
    if (!dirty || S.prev_full || (*dirty)[b]) return true;
    for (int a = a0; a < a1; ++a)
      if (!(job == 0 && S.col_prev[a])) return false;
    return true;
  };
  std::vector<int32_t> items, rest;
  const int nch = (p3 + q - 1) / q;
  for (int b : lb)
    for (int c = 0; c < nch; ++c)
      for (int job = 0; job < 2; ++job) {
        if (!swept(b, c, job)) continue;
        items.insert(items.end(), {b, c, job});
        const HBox &B = t.boxes[b];
        if (!B.leaf)
          for (int ch = 0; ch < B.nchild; ++ch)
            if (!child_swept(B.child[ch], c * q, std::min(p3, (c + 1) * q),
                             job))
              rest.insert(rest.end(), {B.child[ch], c, job});
      }
  S.col_prev = col;
  S.prev_full = all;
  const int64_t ni = (int64_t)items.size(), nr = (int64_t)rest.size();
  if (S.off + ni + nr > (int64_t)ctx->sitems.n)
    return fail(ctx, SKEL_ECAPACITY, "bordered sweep item buffer");
  int32_t *di = ctx->sitems.p + S.off, *dr = di + ni;
  S.off += ni + nr;
  const size_t hb = ctx->hbox.size() * sizeof(DevBox);
  char *ph = static_cast<char *>(pin_take(ctx, hb + (ni + nr) * 4));
  if (!ph) return fail(ctx, SKEL_ENOMEM, "pinned staging buffer");
  std::memcpy(ph, ctx->hbox.data(), hb);
  std::memcpy(ph + hb, items.data(), ni * 4);
  std::memcpy(ph + hb + ni * 4, rest.data(), nr * 4);
  CU(cudaMemcpyAsync(ctx->dbox_sw.p, ph, hb, cudaMemcpyHostToDevice,
                     ctx->st3));
  if (ni + nr)
    CU(cudaMemcpyAsync(di, ph + hb, (ni + nr) * 4, cudaMemcpyHostToDevice,
                       ctx->st3));
  timed_on(ctx, KC_BORDER, ctx->st3, [&] {
    UpJobs j{{ctx->W.p, ctx->Wt.p}, {ctx->UH.p, ctx->QT.p}, {0, 1},
             {ctx->H0.p, ctx->P0.p}, ctx->snap.p};
    launch_snap_restore(ctx->dbox_sw.p, dr, (int)(nr / 3), ctx->dofs.p, j, n2,
                        p3, q, ctx->st3);
    // the mixed form sweeps in FP32 arithmetic over its FP64 factors: the
    // swept columns enter only the preconditioner (the top block's bordering
    // and the back substitution), whose accuracy is the ID tolerance's
    if (ctx->fac32)
      launch_up_items<float, double>(
          ctx->dbox_sw.p, di, (int)(ni / 3), ctx->dofs.p,
          reinterpret_cast<const float *>(ctx->fac.p), ctx->ipool.p, j, n2,
          p3, q, maxn, ctx->dstatus3.p, ctx->st3);
    else if (ctx->id32)
      launch_up_items<double, float>(ctx->dbox_sw.p, di, (int)(ni / 3),
                                     ctx->dofs.p, ctx->fac.p, ctx->ipool.p, j,
                                     n2, p3, q, maxn, ctx->dstatus3.p,
                                     ctx->st3);
    else
      launch_up_items<double, double>(ctx->dbox_sw.p, di, (int)(ni / 3),
                                      ctx->dofs.p, ctx->fac.p, ctx->ipool.p,
                                      j, n2, p3, q, maxn, ctx->dstatus3.p,
                                      ctx->st3);
  });
  if (l == 1) ctx->bord_lv_q = S.lv_q;
  return SKEL_OK;
}

static int factor_all(skel_ctx *ctx, const std::vector<char> *dirty) {
  const Tree &t = ctx->tree;
  int rc;
  if ((rc = upload_level_ids(ctx))) return rc;
  if ((rc = bord_begin(ctx, dirty))) return rc;
  for (int l = t.L(); l >= 1; --l) {
    std::vector<int> work;
    for (int b : t.levels[l])
      if (!dirty || (*dirty)[b]) work.push_back(b);
    double t0 = now_ms();
    if ((rc = compress_level(ctx, l, work))) return rc;
    ctx->lv_ms[l] = now_ms() - t0;
    if ((rc = bord_level(ctx, l))) return rc;
  }
  // a non-dirty level still needs its per-box sizes on the device
  CU(ctx->dbox.ensure(ctx->hbox.size()));
  CU(cudaMemcpyAsync(ctx->dbox.p, ctx->hbox.data(),
                     ctx->hbox.size() * sizeof(DevBox), cudaMemcpyHostToDevice,
                     ctx->st));
  // the sweeps size their shared memory by the largest box of each level,
  // recomputed or reused
  ctx->lv_alln.assign(t.levels.size(), 0);
  for (int l = 1; l <= t.L(); ++l)
    for (int b : t.levels[l])
      ctx->lv_alln[l] = std::max(ctx->lv_alln[l], ctx->hbox[b].n);
  return factor_top(ctx);
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

void skel_default_params(skel_params *o) {
  if (!o) return;
  o->leaf_size = 64;
  o->n_proxy = 64;
  o->proxy_ratio = 1.5;
  o->id_tol = 1e-12;
  o->precision = SKEL_FP64;
  o->gmres_tol = 1e-12;
  o->gmres_maxit = 50;
  o->kernel = SKEL_KERNEL_STOKES;
}

int skel_build_tree(const skel_geom *geom, const skel_params *params,
                    void *cuda_stream, skel_ctx **out) {
  if (!out) return fail(nullptr, SKEL_EINVAL, "out is NULL");
  *out = nullptr;
  if (check_geom_args(geom))
    return fail(nullptr, SKEL_EINVAL, "invalid geometry arguments");
  skel_params prm;
  skel_default_params(&prm);
  if (params) prm = *params;
  if (prm.leaf_size < 1 || prm.n_proxy < 4 || prm.n_proxy > 256 ||
      !(prm.proxy_ratio > 1.0) ||
      !(prm.id_tol >= 0.0) || (prm.precision != SKEL_FP64 &&
                               prm.precision != SKEL_MIXED) ||
      (prm.kernel != SKEL_KERNEL_STOKES && prm.kernel != SKEL_KERNEL_LAPLACE))
    return fail(nullptr, SKEL_EINVAL, "invalid parameters");
  if (prm.kernel == SKEL_KERNEL_LAPLACE && prm.precision != SKEL_FP64)
    return fail(nullptr, SKEL_EINVAL, "the Laplace form is FP64 only");
  std::unique_ptr<skel_ctx> ctx(new skel_ctx());
  ctx->prm = prm;
  ctx->lap = prm.kernel == SKEL_KERNEL_LAPLACE;
  ctx->dpn = ctx->lap ? 1 : 2;
  // The mixed form builds the ID matrices and their Householder updates in
  // FP32 (rank decisions and T solves in FP64) and eliminates in FP64.
  // SKEL_MIXED_FACTORS=fp32 also eliminates and stores the factors in FP32
  // (experimental: on large top-level boxes the FP32 LU and Schur
  // complements spoil the preconditioner).
  ctx->id32 = prm.precision == SKEL_MIXED;
  if (const char *v = std::getenv("SKEL_MIXED_FACTORS"))
    ctx->fac32 = ctx->id32 && std::strcmp(v, "fp32") == 0;
  ctx->st = (cudaStream_t)cuda_stream;
  int rc = load_geometry(ctx.get(), geom);
  if (rc) {
    g_last_error = ctx->err;
    return rc;
  }
  std::string err;
  if (!build_tree(ctx->hx.data(), ctx->hy.data(), ctx->hcomp.data(), ctx->N,
                  prm.leaf_size, ctx->tree, err)) {
    g_last_error = err;
    return SKEL_EINVAL;
  }
  const HBox &R = ctx->tree.boxes[0];
  ctx->root_cx = R.cx;
  ctx->root_cy = R.cy;
  ctx->root_hw = R.hw;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (ctx->dstatus.ensure(4) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->sthi, cudaStreamNonBlocking,
                                   prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->st2, cudaStreamNonBlocking,
                                   prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->st3, cudaStreamNonBlocking,
                                   prio_lo) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork3, cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join3, cudaEventDisableTiming) !=
          cudaSuccess) {
    g_last_error = "CUDA stream/event/allocation setup failed";
    return SKEL_ECUDA;
  }
  if (const char *v = std::getenv("SKEL_SOLVE_GRAPHS"))
    ctx->graphs = std::atoi(v) != 0;
  // boxes above 1.25 leaves of active DOFs go to the clusters by default:
  // a leaf stays on one CTA (the 64-hole quadrant case with leaves of 128
  // nodes: 256-DOF leaves on clusters cost 19 % of its FP64 factorization
  // and 25 % of the mixed one, measured by the autotuner)
  ctx->cluster_min_n =
      std::max(160, (5 * ctx->dpn * ctx->prm.leaf_size + 3) / 4);
  if (const char *v = std::getenv("SKEL_CLUSTER_MIN_N"))
    ctx->cluster_min_n = std::max(1, std::atoi(v));
  *out = ctx.release();
  return SKEL_OK;
}

// Runs a factorization or an update on ctx->sthi: forked from the
// caller's stream on entry, joined back on exit (also on errors).
struct OnPriorityStream {
  skel_ctx *c;
  cudaStream_t user;
  explicit OnPriorityStream(skel_ctx *ctx) : c(ctx), user(ctx->st) {
    cudaEventRecord(c->ev_in, user);
    cudaStreamWaitEvent(c->sthi, c->ev_in, 0);
    c->st = c->sthi;
  }
  ~OnPriorityStream() {
    cudaEventRecord(c->ev_out, c->sthi);
    cudaStreamWaitEvent(user, c->ev_out, 0);
    c->st = user;
  }
};

int skel_factor(skel_ctx *ctx) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  OnPriorityStream on_hi(ctx);
  double t0 = now_ms();
  const double a0 = dev_alloc_ms();
  ctx->wait_ms = 0;
  ctx->host_prep_ms = ctx->host_post_ms = 0;
  drop_graphs(ctx);
  ctx->factored = false;
  const size_t nb = ctx->tree.boxes.size();
  ctx->hbox.assign(nb, DevBox{});
  ctx->hdofs.assign(nb, {});
  ctx->hnear.assign(nb, {});
  box_contents(ctx);
  ctx->fac.used = ctx->ipool.used = ctx->dofs.used = 0;
  ctx->live_fac = 0;
  reset_stats(ctx);
  ctx->bord_full = true;
  int rc = factor_all(ctx, nullptr);
  if (rc) return rc;
  ctx->factored = true;
  ctx->last_dirty = ctx->last_boxes = (int64_t)nb;
  ctx->t_factor_ms = now_ms() - t0;
  ctx->host_factor_ms = ctx->t_factor_ms - ctx->wait_ms;
  ctx->alloc_ms = dev_alloc_ms() - a0;
  return SKEL_OK;
}

// The update of Sec. 2.8 for a new geometry.  old_of_new (nullptr: the
// identity, same N) gives for every new node its id before the update, or
// -1 for a new node; ids that are kept must stay increasing.  Boxes whose
// subtree content (node identities and geometry), children and near
// owners are unchanged keep their factors, with their DOF lists renumbered;
// the others are recompressed, and the top block is redone.
static int update_impl(skel_ctx *ctx, const skel_geom *new_geom,
                       const std::vector<int64_t> *old_of_new, double t0) {
  OnPriorityStream on_hi(ctx);
  const double a0 = dev_alloc_ms();
  drop_graphs(ctx);
  const int64_t old_N = ctx->N;
  // keep the old tree and records
  Tree old_tree = ctx->tree;
  std::vector<DevBox> old_box = ctx->hbox;
  std::vector<std::vector<int32_t>> old_dofs = ctx->hdofs;
  std::vector<std::vector<int>> old_near = ctx->hnear;
  std::vector<uint64_t> old_content = ctx->content;
  const std::vector<double> old_cent = ctx->hcent;
  const int old_p = ctx->p;
  int rc = load_geometry(ctx, new_geom);
  if (rc) return rc;
  // bordered columns: a renumbering or a new hole count sweeps everything
  // again; otherwise the H columns of a hole whose centre moved change at
  // every node (the Psi columns depend on the nodes alone)
  ctx->bord_full = old_of_new != nullptr || old_p != ctx->p ||
                   old_cent.size() != ctx->hcent.size();
  ctx->bord_col_changed.assign(3 * (size_t)ctx->p, 0);
  if (!ctx->bord_full)
    for (int i = 0; i < ctx->p; ++i)
      if (old_cent[2 * i] != ctx->hcent[2 * i] ||
          old_cent[2 * i + 1] != ctx->hcent[2 * i + 1])
        for (int a = 0; a < 3; ++a) ctx->bord_col_changed[3 * i + a] = 1;
  for (int64_t i = 0; i < ctx->N; ++i)
    if (!(std::fabs(ctx->hx[i] - ctx->root_cx) <= ctx->root_hw &&
          std::fabs(ctx->hy[i] - ctx->root_cy) <= ctx->root_hw))
      return fail(ctx, SKEL_EINVAL, "node outside the root box");
  build_tree_root(ctx->hx.data(), ctx->hy.data(), ctx->N, ctx->prm.leaf_size,
                  ctx->root_cx, ctx->root_cy, ctx->root_hw, ctx->tree);
  const Tree &t = ctx->tree;
  const size_t nb = t.boxes.size();
  // identities: the old id of a kept node, a fresh one (>= old_N) for a new
  std::vector<int64_t> ident;
  std::vector<int32_t> new_of_old;
  if (old_of_new) {
    ident.resize(ctx->N);
    new_of_old.assign(old_N, -1);
    for (int64_t j = 0; j < ctx->N; ++j) {
      const int64_t o = (*old_of_new)[j];
      ident[j] = o >= 0 ? o : old_N + j;
      if (o >= 0) new_of_old[o] = (int32_t)j;
    }
  }
  box_contents(ctx, old_of_new ? ident.data() : nullptr);
  ctx->hbox.assign(nb, DevBox{});
  ctx->hdofs.assign(nb, {});
  ctx->hnear.assign(nb, {});
  // Sec. 2.8 marking: a box is recompressed when it is new, its subtree
  // content changed, a child was recompressed, or a near owner changed
  // (or appeared / disappeared from its proxy disk).
  std::vector<char> dirty(nb, 0);
  std::vector<char> changed(nb, 0);
  std::vector<int> near;
  auto old_id = [&](int b) -> int {
    const HBox &B = t.boxes[b];
    auto it = old_tree.key2id.find(box_key(B.depth, B.ix, B.iy));
    return it == old_tree.key2id.end() ? -1 : it->second;
  };
  std::vector<int> reused;
  for (int l = t.L(); l >= 1; --l) {
    // in_changed for the owners at the start of level l
    for (size_t o = 0; o < nb; ++o) {
      const HBox &X = t.boxes[o];
      if (!(X.depth == l || (X.leaf && X.depth < l))) continue;
      int ob = old_id((int)o);
      bool ch = ob < 0 || old_content[ob] != ctx->content[o] ||
                old_tree.boxes[ob].leaf != X.leaf;
      if (!ch && X.depth == l && !X.leaf)
        for (int c = 0; c < X.nchild; ++c) ch = ch || dirty[X.child[c]];
      changed[o] = ch;
    }
    for (int b : t.levels[l]) {
      near_owners(t, b, l, ctx->prm.proxy_ratio, near);
      int ob = old_id(b);
      bool d = changed[b] || ob < 0;
      for (int o : near) d = d || changed[o];
      if (!d) {
        const auto &on = old_near[ob];
        if (on.size() != near.size()) {
          d = true;
        } else {
          for (size_t i = 0; i < near.size() && !d; ++i) {
            const HBox &A = t.boxes[near[i]];
            const HBox &Bo = old_tree.boxes[on[i]];
            d = A.depth != Bo.depth || A.ix != Bo.ix || A.iy != Bo.iy;
          }
        }
      }
      dirty[b] = d;
      if (!d) {
        ctx->hbox[b] = old_box[ob];
        ctx->hdofs[b] = old_dofs[ob];
        ctx->hnear[b] = near;
        reused.push_back(b);
      }
    }
  }
  int64_t nd = 0;
  for (size_t b = 1; b < nb; ++b) nd += dirty[b];
  // compact the factor arenas from time to time: a full refactor gives the
  // identical factorization
  bool full = ctx->fac.used > 3 * std::max<int64_t>(ctx->live_fac, 1);
  if (old_of_new && !full && !reused.empty()) {
    // renumber the kept boxes' DOF lists (host copies and their slices of
    // the device arena) to the new node ids
    std::vector<int32_t> arena(ctx->dofs.used);
    if (!arena.empty()) {
      CU(sync_st(ctx));
      CU(cudaMemcpy(arena.data(), ctx->dofs.p, arena.size() * sizeof(int32_t),
                    cudaMemcpyDeviceToHost));
    }
    for (int b : reused) {
      auto &v = ctx->hdofs[b];
      for (auto &d : v) {
        const int32_t j = new_of_old[dof_node(ctx, d)];
        if (j < 0) return fail(ctx, SKEL_EINVAL, "kept box lost a node");
        d = ctx->dpn == 2 ? 2 * j + (d & 1) : j;
      }
      std::copy(v.begin(), v.end(), arena.begin() + ctx->hbox[b].dof_off);
    }
    if (!arena.empty())
      CU(cudaMemcpyAsync(ctx->dofs.p, arena.data(),
                         arena.size() * sizeof(int32_t),
                         cudaMemcpyHostToDevice, ctx->st));
    CU(sync_st(ctx));  // the host copy goes out of scope
  }
  reset_stats(ctx);
  if (full) {
    ctx->fac.used = ctx->ipool.used = ctx->dofs.used = 0;
    ctx->live_fac = 0;
    ctx->hbox.assign(nb, DevBox{});
    ctx->hdofs.assign(nb, {});
    rc = factor_all(ctx, nullptr);
  } else {
    rc = factor_all(ctx, &dirty);
  }
  if (rc) {
    ctx->factored = false;
    return rc;
  }
  // digests under the new numbering, for the next update
  if (old_of_new) box_contents(ctx);
  ctx->factored = true;
  ctx->last_dirty = nd;
  ctx->last_boxes = (int64_t)nb - 1;
  ctx->t_update_ms = now_ms() - t0;
  ctx->host_update_ms = ctx->t_update_ms - ctx->wait_ms;
  ctx->alloc_ms = dev_alloc_ms() - a0;
  return SKEL_OK;
}

int skel_update_moved_nodes(skel_ctx *ctx, int64_t n_moved,
                            const int64_t *node_ids,
                            const skel_geom *new_geom) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (!ctx->factored) return fail(ctx, SKEL_ESTATE, "update before factor");
  if (check_geom_args(new_geom) || new_geom->N != ctx->N ||
      new_geom->p != ctx->p || n_moved < 0 || (n_moved > 0 && !node_ids))
    return fail(ctx, SKEL_EINVAL, "invalid update arguments");
  double t0 = now_ms();
  ctx->wait_ms = 0;
  ctx->host_prep_ms = ctx->host_post_ms = 0;
  std::vector<int64_t> ids(n_moved);
  if (n_moved)
    CU(cudaMemcpy(ids.data(), node_ids, n_moved * sizeof(int64_t),
                  cudaMemcpyDefault));
  for (int64_t j : ids)
    if (j < 0 || j >= ctx->N)
      return fail(ctx, SKEL_EINVAL, "moved node id out of range");
  return update_impl(ctx, new_geom, nullptr, t0);
}

int skel_update_geometry(skel_ctx *ctx, const skel_geom *new_geom,
                         const int64_t *old_id) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (!ctx->factored) return fail(ctx, SKEL_ESTATE, "update before factor");
  if (check_geom_args(new_geom) || !old_id)
    return fail(ctx, SKEL_EINVAL, "invalid update arguments");
  double t0 = now_ms();
  ctx->wait_ms = 0;
  ctx->host_prep_ms = ctx->host_post_ms = 0;
  std::vector<int64_t> map(new_geom->N);
  if (new_geom->N)
    CU(cudaMemcpy(map.data(), old_id, new_geom->N * sizeof(int64_t),
                  cudaMemcpyDefault));
  int64_t last = -1;
  for (int64_t o : map) {
    if (o < -1 || o >= ctx->N || (o >= 0 && o <= last))
      return fail(ctx, SKEL_EINVAL,
                  "old_id must be -1 or increasing ids of the old geometry");
    if (o >= 0) last = o;
  }
  return update_impl(ctx, new_geom, &map, t0);
}

// The factored solve x <- (V X_D^{-1} U) x with the bordered top block
// (Eq. solution, Eq. partition), in place on device columns x (ld ldf);
// adjoint applies the transposed factors in reverse order.  Enqueued on
// the context's stream, no synchronisation.
static int fsolve(skel_ctx *ctx, int nrhs, double *x, int adjoint) {
  const Tree &t = ctx->tree;
  const int64_t n2 = ndof(ctx);
  const int p3 = nbord(ctx);
  const int64_t ldf = n2 + p3;
  const int ldt = ctx->ldt;
  CU(ctx->rhs_top.ensure((size_t)ldt * nrhs + 1));
  const int nchunk = top_rhs_chunks(n2, p3, nrhs);
  CU(ctx->partial.ensure((size_t)nchunk * nrhs * std::max(p3, 1) + 1));
  timed(ctx, KC_UP, [&] {
    for (int l = t.L(); l >= 1; --l)
      sweep_up(ctx, l, x, ldf, nrhs, nullptr, adjoint);
  });
  timed(ctx, KC_TOPSOLVE, [&] {
    launch_top_rhs(x, ldf, nrhs, ctx->droot_act.p, ctx->s,
                   adjoint ? ctx->UH.p : ctx->QT.p, n2, p3, ctx->rmask.p, n2,
                   x + n2, ldf, ctx->partial.p, ctx->rhs_top.p, ldt, ctx->st);
    launch_dense_lu_solve(ctx->top.p, ldt, ldt, ctx->top_piv.p,
                          ctx->rhs_top.p, ldt, nrhs, adjoint, ctx->st);
    launch_top_back(x, ldf, nrhs, ctx->droot_act.p, ctx->s,
                    adjoint ? ctx->Wt.p : ctx->W.p, n2, p3, ctx->rmask.p, n2,
                    ctx->rhs_top.p, ldt, ctx->st);
  });
  timed(ctx, KC_DOWN, [&] {
    for (int l = 1; l <= t.L(); ++l) sweep_down(ctx, l, x, ldf, nrhs, adjoint);
  });
  // factor bytes read by the sweeps (T and Z or Y up, LU up, Y or Z and T
  // down) plus the gathered vector entries
  const double esz = ctx->fac32 ? 4.0 : 8.0;
  double up = 0.0, down = 0.0;
  for (size_t b = 1; b < ctx->hbox.size(); ++b) {
    const double k = ctx->hbox[b].k, r = ctx->hbox[b].n - ctx->hbox[b].k;
    up += esz * (2 * k * r + r * r);
    down += esz * (2 * k * r);
  }
  ctx->kst[KC_UP].bytes += up + 8.0 * 2 * n2 * nrhs;
  ctx->kst[KC_DOWN].bytes += down + 8.0 * 2 * n2 * nrhs;
  CU(cudaGetLastError());
  return SKEL_OK;
}

// One-column factored solve in place on the device column x.  The launches
// of fsolve are fixed once the factorization is: the first call runs them
// directly on the graph's column (which also sizes every buffer they use),
// then records them as a CUDA graph; later calls copy x in, replay the
// graph (one launch instead of about 20) and copy the result out.  With
// per-kernel timing on (events between the launches) it runs directly.
static int fsolve1(skel_ctx *ctx, double *x, int adjoint) {
  if (ctx->timing || !ctx->graphs) return fsolve(ctx, 1, x, adjoint);
  const int64_t ldf = nsys(ctx);
  CU(ctx->gsol.ensure((size_t)ldf));
  double *gx = ctx->gsol.p;
  CU(cudaMemcpyAsync(gx, x, ldf * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->st));
  if (ctx->sgraph[adjoint]) {
    CU(cudaGraphLaunch(ctx->sgraph[adjoint], ctx->st));
    note_launches((int)ctx->sgraph_launches[adjoint]);
  } else {
    int rc = fsolve(ctx, 1, gx, adjoint);
    if (rc) return rc;
    // record the same launches (nothing runs while capturing); the
    // statistics and the launch counter must not see them
    KStat saved[KC_N];
    std::copy(ctx->kst, ctx->kst + KC_N, saved);
    const int64_t l0 = g_launches.load();
    cudaGraph_t graph = nullptr;
    cudaError_t e =
        cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = fsolve(ctx, 1, gx, adjoint);
      e = cudaStreamEndCapture(ctx->st, &graph);
    }
    const int64_t lcap = g_launches.load() - l0;
    g_launches -= lcap;
    std::copy(saved, saved + KC_N, ctx->kst);
    cudaGraphExec_t exec = nullptr;
    if (rc == SKEL_OK && e == cudaSuccess && graph)
      e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != SKEL_OK || e != cudaSuccess || !exec) {
      // capture unsupported here: keep solving without graphs
      (void)cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      ctx->graphs = false;
    } else {
      ctx->sgraph[adjoint] = exec;
      ctx->sgraph_launches[adjoint] = lcap;
    }
  }
  CU(cudaMemcpyAsync(x, gx, ldf * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->st));
  return SKEL_OK;
}

// y <- A x or A^T x with the FP64 operator (device columns, ld ldf)
static int op_apply(skel_ctx *ctx, const double *x, double *y, int adjoint) {
  const int64_t ldf = nsys(ctx);
  CU(ctx->dlscr.ensure(dl_scratch(ctx->N, 1, ctx->N)));
  timed(ctx, KC_MATVEC, [&] {
    if (adjoint)
      launch_matvec_adjoint(ctx->g, 1, x, y, ldf, ctx->dlscr.p, ctx->st);
    else
      launch_matvec(ctx->g, 1, x, y, ldf, ctx->dlscr.p, ctx->st);
  });
  ctx->kst[KC_MATVEC].flops += kPairFlops * (double)ctx->N * ctx->N;
  return SKEL_OK;
}

// y <- A x with the double-layer sums in double-float arithmetic (the
// operator of the GMRES iterations; not used for the adjoint)
static int op_apply_fast(skel_ctx *ctx, const double *x, double *y,
                         int adjoint) {
  const int nblk = (int)(ctx->hdlf_blk.size() / 2);
  CU(ctx->dlfscr.ensure(dlf_scratch(ctx->N, nblk)));
  timed(ctx, KC_MATVEC_DF, [&] {
    if (adjoint)
      launch_matvec_fast_adjoint(ctx->g, x, y, ctx->dlf_blk.p, nblk,
                                 ctx->dlfscr.p, ctx->st);
    else
      launch_matvec_fast(ctx->g, x, y, ctx->dlf_blk.p, nblk, ctx->dlfscr.p,
                         ctx->st);
  });
  ctx->kst[KC_MATVEC_DF].flops += kPairFlops * (double)ctx->N * ctx->N;
  return SKEL_OK;
}

// host copy of a few device doubles (synchronises the stream)
static int fetch(skel_ctx *ctx, const double *d, double *h, int n) {
  CU(sync_st(ctx));
  CU(cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->st));
  CU(sync_st(ctx));
  return SKEL_OK;
}

// Restarted GMRES with right preconditioning by the factored solve, on the
// FP64 operator (the low-precision factorization used as a preconditioner,
// Eq. kinv remark).  Column b (device) -> x (device).  Orthogonalisation by
// classical Gram-Schmidt applied twice.
static int gmres_column(skel_ctx *ctx, const double *b, double *x, int adjoint,
                        int &iters, double &relres) {
  const int64_t n = nsys(ctx);
  const int m = 30;
  const double tol = ctx->prm.gmres_tol;
  const int maxit = std::max(1, ctx->prm.gmres_maxit);
  CU(ctx->gmV.ensure((size_t)n * (m + 1)));
  CU(ctx->gmZ.ensure((size_t)n * m));
  CU(ctx->gmw.ensure((size_t)n));
  CU(ctx->gmdot.ensure(multidot_scratch() + 4 * 64));
  double *V = ctx->gmV.p, *Z = ctx->gmZ.p, *w = ctx->gmw.p;
  // dres: two Gram-Schmidt passes' coefficients and a norm (64 each), so
  // one host round trip per Krylov step fetches all three
  double *part = ctx->gmdot.p, *dres = part + multidot_scratch();
  double *dcoef = dres + 3 * 64;
  int rc;
  auto dot = [&](const double *u, const double *v, double &out) -> int {
    launch_multidot(u, v, n, 1, n, part, dres, ctx->st);
    return fetch(ctx, dres, &out, 1);
  };
  double bn2 = 0.0;
  if ((rc = dot(b, b, bn2))) return rc;
  const double bnorm = std::sqrt(bn2);
  iters = 0;
  relres = 0.0;
  if (bnorm == 0.0) {
    CU(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->st));
    return SKEL_OK;
  }
  // x0 = M^{-1} b
  CU(cudaMemcpyAsync(x, b, n * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->st));
  if ((rc = fsolve1(ctx, x, adjoint))) return rc;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1),
      hcol(m + 1), hbuf(3 * 64);
  // Krylov products use the double-float operator (or its transpose) when
  // available.  The residual that decides convergence is the double-float
  // one when the tolerance is at least kDfCheckTol (50x the operator's
  // 2e-13 relative accuracy), else, or on request, the FP64 one; an FP64
  // residual that fails after a cycle switches the rest to FP64.
  bool fast = !ctx->hdlf_blk.empty();
  const bool df_check = fast && !ctx->gmres_fp64_check && tol >= kDfCheckTol;
  ctx->last_check_df = df_check;
  ctx->last_check_rec = false;
  bool check = !fast;  // the residual at the top of the loop is FP64
  int cycles = 0;
  auto apply = [&](const double *in, double *out, bool exact) -> int {
    return exact ? op_apply(ctx, in, out, adjoint)
                 : op_apply_fast(ctx, in, out, adjoint);
  };
  while (true) {
    // r = b - A x, stored in V[:, 0]
    if ((rc = apply(x, V, check))) return rc;
    launch_axpby(1.0, b, -1.0, V, n, ctx->st);
    double r2 = 0.0;
    if ((rc = dot(V, V, r2))) return rc;
    const double beta = std::sqrt(r2);
    relres = beta / bnorm;
    if (cycles == 0) ctx->last_relres0 = relres;  // after x0 = M^{-1} b
    if (!check) {
      if (relres <= tol || iters >= maxit) {
        if (df_check) break;
        check = true;  // confirm with the FP64 operator
        continue;
      }
    } else {
      if (relres <= tol || iters >= maxit) break;
      if (cycles > 0) fast = false;
    }
    // the inner target leaves room for the double-float operator's error
    const double tol_in = fast ? 0.25 * tol : tol;
    launch_axpby(1.0 / beta, V, 0.0, V, n, ctx->st);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    bool inner_done = false;
    for (; j < m && iters < maxit; ++j, ++iters) {
      double *zj = Z + (int64_t)j * n, *vj = V + (int64_t)j * n;
      CU(cudaMemcpyAsync(zj, vj, n * sizeof(double), cudaMemcpyDeviceToDevice,
                         ctx->st));
      if ((rc = fsolve1(ctx, zj, adjoint))) return rc;
      if ((rc = apply(zj, w, !fast))) return rc;
      // two passes of classical Gram-Schmidt against V[:, 0..j], then the
      // norm of what is left; all three read back at once
      for (int pass = 0; pass < 2; ++pass) {
        launch_multidot(w, V, n, j + 1, n, part, dres + 64 * pass, ctx->st);
        launch_combine(w, 1.0, V, n, dres + 64 * pass, -1.0, j + 1, n,
                       ctx->st);
      }
      launch_multidot(w, w, n, 1, n, part, dres + 128, ctx->st);
      if ((rc = fetch(ctx, dres, hbuf.data(), 129))) return rc;
      for (int i = 0; i <= j; ++i) hcol[i] = hbuf[i] + hbuf[64 + i];
      hcol[j + 1] = std::sqrt(hbuf[128]);
      if (hcol[j + 1] > 0.0)
        launch_axpby(1.0 / hcol[j + 1], w, 0.0, V + (int64_t)(j + 1) * n, n,
                     ctx->st);
      // Givens rotations on the new column of the Hessenberg matrix
      for (int i = 0; i < j; ++i) {
        const double a = hcol[i], c = hcol[i + 1];
        hcol[i] = cs[i] * a + sn[i] * c;
        hcol[i + 1] = -sn[i] * a + cs[i] * c;
      }
      const double a = hcol[j], c = hcol[j + 1];
      const double rr = std::hypot(a, c);
      cs[j] = rr > 0.0 ? a / rr : 1.0;
      sn[j] = rr > 0.0 ? c / rr : 0.0;
      hcol[j] = rr;
      hcol[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      if (std::fabs(gv[j + 1]) / bnorm <= tol_in) {
        ++j;
        ++iters;
        inner_done = true;
        break;
      }
    }
    ++cycles;
    check = !df_check;
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = gv[i];
      for (int l = i + 1; l < j; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    if (j > 0) {
      CU(cudaMemcpyAsync(dcoef, y.data(), j * sizeof(double),
                         cudaMemcpyHostToDevice, ctx->st));
      launch_combine(x, 1.0, Z, n, dcoef, 1.0, j, n, ctx->st);
    }
    // With the double-float operator deciding convergence, a cycle whose
    // residual recurrence met the inner target ends the solve without one
    // more operator apply: b - A x_j = r_0 - A Z y is V_{j+1}(beta e_1 -
    // Hbar y) by the Arnoldi relation of that same operator (FP64 vectors,
    // Gram-Schmidt twice), whose norm is |g_{j+1}|; a fresh apply of the
    // same operator would add only its own rounding.  The FP64 test, and
    // a cycle ended by the iteration limit, still apply the operator.
    if (df_check && inner_done) {
      relres = std::fabs(gv[j]) / bnorm;
      ctx->last_check_rec = true;
      break;
    }
  }
  return SKEL_OK;
}

static int solve_impl(skel_ctx *ctx, int32_t nrhs, const double *f,
                      double *out, int adjoint) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (!ctx->factored) return fail(ctx, SKEL_ESTATE, "solve before factor");
  if (nrhs < 0 || nrhs > kMaxCols || (nrhs > 0 && (!f || !out)))
    return fail(ctx, SKEL_EINVAL, "invalid solve arguments");
  if (nrhs == 0) return SKEL_OK;
  double t0 = now_ms();
  ctx->wait_ms = 0;
  ctx->host_prep_ms = ctx->host_post_ms = 0;
  const int64_t ldf = nsys(ctx);
  CU(ctx->work.ensure((size_t)ldf * nrhs));
  CU(cudaMemcpyAsync(ctx->work.p, f, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaMemsetAsync(ctx->dstatus.p, 0, sizeof(int), ctx->st));
  int rc;
  ctx->last_iters = 0;
  ctx->last_relres = 0.0;
  if (!is_mixed(ctx)) {
    if ((rc = nrhs == 1 ? fsolve1(ctx, ctx->work.p, adjoint)
                        : fsolve(ctx, nrhs, ctx->work.p, adjoint)))
      return rc;
    CU(cudaMemcpyAsync(out, ctx->work.p, (size_t)ldf * nrhs * sizeof(double),
                       cudaMemcpyDefault, ctx->st));
  } else {
    CU(ctx->gmx.ensure((size_t)ldf));
    for (int q = 0; q < nrhs; ++q) {
      int it = 0;
      double rr = 0.0;
      if ((rc = gmres_column(ctx, ctx->work.p + (int64_t)q * ldf, ctx->gmx.p,
                             adjoint, it, rr)))
        return rc;
      ctx->last_iters = std::max(ctx->last_iters, it);
      if (!(rr <= ctx->last_relres)) ctx->last_relres = rr;  // keeps a NaN
      CU(cudaMemcpyAsync(out + (int64_t)q * ldf, ctx->gmx.p,
                         ldf * sizeof(double), cudaMemcpyDefault, ctx->st));
    }
  }
  int status = 0;
  CU(sync_st(ctx));
  CU(cudaMemcpyAsync(&status, ctx->dstatus.p, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->st));
  CU(sync_st(ctx));
  resolve_timing(ctx);
  if (status != 0) return fail(ctx, status, "a sweep kernel rejected a box");
  ctx->t_solve_ms = now_ms() - t0;
  ctx->host_solve_ms = ctx->t_solve_ms - ctx->wait_ms;
  if (is_mixed(ctx) && !(ctx->last_relres <= ctx->prm.gmres_tol)) {
    char buf[96];
    std::snprintf(buf, sizeof buf,
                  "GMRES stopped at relative residual %.3e after %d iterations",
                  ctx->last_relres, ctx->last_iters);
    return fail(ctx, SKEL_ENOCONV, buf);
  }
  return SKEL_OK;
}

int skel_solve(skel_ctx *ctx, int32_t nrhs, const double *f, double *out) {
  return solve_impl(ctx, nrhs, f, out, 0);
}

int skel_solve_adjoint(skel_ctx *ctx, int32_t nrhs, const double *g,
                       double *out) {
  return solve_impl(ctx, nrhs, g, out, 1);
}

int skel_eval_velocity(skel_ctx *ctx, int32_t nrhs, const double *sol,
                       int64_t nt, const double *tx, const double *ty,
                       double *u) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (nrhs < 0 || nrhs > kMaxCols || nt < 0 ||
      (nrhs > 0 && nt > 0 && (!sol || !tx || !ty || !u)))
    return fail(ctx, SKEL_EINVAL, "invalid eval arguments");
  if (nrhs == 0 || nt == 0) return SKEL_OK;
  const int64_t ldf = nsys(ctx);
  CU(ctx->vin.ensure((size_t)ldf * nrhs + 2 * nt));
  CU(ctx->vout.ensure((size_t)2 * nt * nrhs));
  double *dsol = ctx->vin.p, *dtx = dsol + ldf * nrhs, *dty = dtx + nt;
  CU(cudaMemcpyAsync(dsol, sol, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaMemcpyAsync(dtx, tx, nt * sizeof(double), cudaMemcpyDefault, ctx->st));
  CU(cudaMemcpyAsync(dty, ty, nt * sizeof(double), cudaMemcpyDefault, ctx->st));
  CU(ctx->dlscr.ensure(dl_scratch(nt, nrhs, ctx->N)));
  timed(ctx, KC_EVAL, [&] {
    if (ctx->lap)
      launch_lap_potential(ctx->g, nrhs, dsol, ldf, nt, dtx, dty, ctx->vout.p,
                           ctx->st);
    else
      launch_eval_velocity(ctx->g, nrhs, dsol, ldf, nt, dtx, dty,
                           ctx->vout.p, ctx->dlscr.p, ctx->st);
  });
  ctx->kst[KC_EVAL].flops += kPairFlops * (double)ctx->N * nt * nrhs;
  CU(cudaGetLastError());
  const int comps = ctx->lap ? 1 : 2;  // potential, or velocity components
  CU(cudaMemcpyAsync(u, ctx->vout.p, (size_t)comps * nt * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

// Allocation-free variant of skel_eval_velocity: device arrays only, no
// staging buffers, no growable scratch, no timing events.
int skel_eval_velocity_noalloc(skel_ctx *ctx, int32_t nrhs, const double *sol,
                               int64_t nt, const double *tx, const double *ty,
                               double *u) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (nrhs < 0 || nt < 0 || (nrhs > 0 && nt > 0 && (!sol || !tx || !ty || !u)))
    return fail(ctx, SKEL_EINVAL, "invalid eval arguments");
  if (nrhs == 0 || nt == 0) return SKEL_OK;
  if (nrhs > kMaxCols)  // one grid row of the launch per right-hand side
    return fail(ctx, SKEL_EINVAL,
                "skel_eval_velocity_noalloc: nrhs may be at most 65535");
  const int64_t max_cols = kNoallocScratchDoubles / 2;
  if (nt > max_cols / nrhs) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "skel_eval_velocity_noalloc: nt * nrhs = %lld exceeds the "
                  "limit of %lld set by its static %lld-byte scratch",
                  (long long)nt * nrhs, (long long)max_cols,
                  (long long)(kNoallocScratchDoubles * sizeof(double)));
    return fail(ctx, SKEL_ECAPACITY, buf);
  }
  const void *ptrs[4] = {sol, tx, ty, u};
  const char *names[4] = {"sol", "tx", "ty", "u"};
  for (int i = 0; i < 4; ++i) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptrs[i]);
    if (e != cudaSuccess || (at.type != cudaMemoryTypeDevice &&
                             at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(ctx, SKEL_EINVAL,
                  std::string("skel_eval_velocity_noalloc: ") + names[i] +
                      " is not device memory (this call stages nothing)");
    }
  }
  const int64_t ldf = nsys(ctx);
  std::string err;
  const int rc = launch_eval_velocity_noalloc(ctx->g, nrhs, sol, ldf, nt, tx,
                                              ty, u, ctx->st, err);
  if (rc != SKEL_OK)
    return fail(ctx, rc, "skel_eval_velocity_noalloc: " + err);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->st));
  return SKEL_OK;
}

int skel_grad_bilinear(skel_ctx *ctx, const double *z, const double *s,
                       double *g) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (!z || !s || !g) return fail(ctx, SKEL_EINVAL, "invalid gradient arguments");
  const int64_t N = ctx->N, ldf = nsys(ctx), ng = 6 * N + 2 * ctx->p;
  CU(ctx->vin.ensure((size_t)2 * ldf));
  CU(ctx->vout.ensure((size_t)ng));
  CU(ctx->gscr.ensure(grad_scratch(N, N)));
  CU(cudaMemcpyAsync(ctx->vin.p, z, ldf * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  CU(cudaMemcpyAsync(ctx->vin.p + ldf, s, ldf * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  timed(ctx, KC_GRAD, [&] {
    launch_grad_bilinear(ctx->g, ctx->gdx.p, ctx->gdy.p, ctx->gddx.p,
                         ctx->gddy.p, ctx->gdt.p, ctx->vin.p, ctx->vin.p + ldf,
                         ctx->gscr.p, ctx->vout.p, ctx->st);
  });
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(g, ctx->vout.p, ng * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

int skel_grad_velocity(skel_ctx *ctx, const double *s, int64_t nt,
                       const double *tx, const double *ty, const double *ubar,
                       double *gs, double *g) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (nt < 0 || !s || !gs || !g || (nt > 0 && (!tx || !ty || !ubar)))
    return fail(ctx, SKEL_EINVAL, "invalid gradient arguments");
  const int64_t N = ctx->N, ldf = nsys(ctx), ng = 6 * N + 2 * ctx->p;
  CU(ctx->vin.ensure((size_t)ldf + 4 * nt + 1));
  CU(ctx->vout.ensure((size_t)ldf + ng));
  CU(ctx->gscr.ensure(grad_scratch(N, nt)));
  double *ds = ctx->vin.p, *dtx = ds + ldf, *dty = dtx + nt, *dub = dty + nt;
  CU(cudaMemcpyAsync(ds, s, ldf * sizeof(double), cudaMemcpyDefault, ctx->st));
  if (nt) {
    CU(cudaMemcpyAsync(dtx, tx, nt * sizeof(double), cudaMemcpyDefault,
                       ctx->st));
    CU(cudaMemcpyAsync(dty, ty, nt * sizeof(double), cudaMemcpyDefault,
                       ctx->st));
    CU(cudaMemcpyAsync(dub, ubar, 2 * nt * sizeof(double), cudaMemcpyDefault,
                       ctx->st));
  }
  double *dgs = ctx->vout.p, *dg = dgs + ldf;
  CU(cudaMemsetAsync(dgs, 0, ldf * sizeof(double), ctx->st));
  CU(cudaMemsetAsync(dg, 0, ng * sizeof(double), ctx->st));
  if (nt)
    timed(ctx, KC_GRAD, [&] {
      launch_grad_velocity(ctx->g, ctx->gdx.p, ctx->gdy.p, ctx->gdt.p, ds, nt,
                           dtx, dty, dub, ctx->gscr.p, dgs, dg, ctx->st);
    });
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(gs, dgs, ldf * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  CU(cudaMemcpyAsync(g, dg, ng * sizeof(double), cudaMemcpyDefault, ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

// J = sum_t |u(x_t)|^2 of the velocity of s = A^{-1} f; s is returned.
int skel_velocity_energy(skel_ctx *ctx, const double *f, int64_t nt,
                         const double *tx, const double *ty, double *J,
                         double *s) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (nt < 0 || !f || !J || !s || (nt > 0 && (!tx || !ty)))
    return fail(ctx, SKEL_EINVAL, "invalid energy arguments");
  const int64_t ldf = nsys(ctx);
  CU(ctx->escr.ensure((size_t)ldf + 2 * nt + 64 + multidot_scratch()));
  double *ds = ctx->escr.p, *du = ds + ldf, *dJ = du + 2 * nt,
         *part = dJ + 64;
  int rc = skel_solve(ctx, 1, f, ds);
  if (rc) return rc;
  *J = 0.0;
  if (nt > 0) {
    if ((rc = skel_eval_velocity(ctx, 1, ds, nt, tx, ty, du))) return rc;
    launch_multidot(du, du, 2 * nt, 1, 2 * nt, part, dJ, ctx->st);
    CU(cudaMemcpyAsync(J, dJ, sizeof(double), cudaMemcpyDefault, ctx->st));
  }
  CU(cudaMemcpyAsync(s, ds, ldf * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  return SKEL_OK;
}

// dJ/dgeometry of J = sum_t |E s|^2 at the solution s of A s = f (f not
// depending on the geometry) by the adjoint method: ubar = 2 E s,
// (gs, gE) from the velocity derivative, A^T z = gs, gA = d(z^T A s), and
// g = gE - gA.
int skel_velocity_energy_gradient(skel_ctx *ctx, const double *s, int64_t nt,
                                  const double *tx, const double *ty,
                                  double *g) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (!ctx->factored)
    return fail(ctx, SKEL_ESTATE, "energy gradient before factor");
  if (nt < 0 || !s || !g || (nt > 0 && (!tx || !ty)))
    return fail(ctx, SKEL_EINVAL, "invalid energy-gradient arguments");
  const int64_t ldf = nsys(ctx), ng = 6 * ctx->N + 2 * ctx->p;
  // [s | u, ubar | gs | z | gE | gA]
  CU(ctx->escr.ensure((size_t)3 * ldf + 4 * nt + 2 * ng + 1));
  double *ds = ctx->escr.p, *du = ds + ldf, *dub = du + 2 * nt,
         *dgs = dub + 2 * nt, *dz = dgs + ldf, *dgE = dz + ldf,
         *dgA = dgE + ng;
  CU(cudaMemcpyAsync(ds, s, ldf * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  int rc;
  if (nt > 0) {
    if ((rc = skel_eval_velocity(ctx, 1, ds, nt, tx, ty, du))) return rc;
    launch_axpby(2.0, du, 0.0, dub, 2 * nt, ctx->st);
  }
  if ((rc = skel_grad_velocity(ctx, ds, nt, tx, ty, dub, dgs, dgE)))
    return rc;
  if ((rc = skel_solve_adjoint(ctx, 1, dgs, dz))) return rc;
  if ((rc = skel_grad_bilinear(ctx, dz, ds, dgA))) return rc;
  launch_axpby(-1.0, dgA, 1.0, dgE, ng, ctx->st);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(g, dgE, ng * sizeof(double), cudaMemcpyDefault,
                     ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  return SKEL_OK;
}

int skel_point_force_rhs(skel_ctx *ctx, int32_t nrhs, int32_t ns,
                         const double *src_xy, const double *src_f,
                         int32_t holes_zero, double *f) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (nrhs < 0 || nrhs > kMaxCols || ns < 0 ||
      (nrhs > 0 && (!f || (ns > 0 && (!src_xy || !src_f)))))
    return fail(ctx, SKEL_EINVAL, "invalid point-force arguments");
  if (nrhs == 0) return SKEL_OK;
  const int64_t ldf = nsys(ctx);
  const size_t nsrc = (size_t)2 * nrhs * ns;
  CU(ctx->vin.ensure(2 * nsrc + 1));
  CU(ctx->vout.ensure((size_t)ldf * nrhs));
  if (nsrc) {
    CU(cudaMemcpyAsync(ctx->vin.p, src_xy, nsrc * sizeof(double),
                       cudaMemcpyDefault, ctx->st));
    CU(cudaMemcpyAsync(ctx->vin.p + nsrc, src_f, nsrc * sizeof(double),
                       cudaMemcpyDefault, ctx->st));
  }
  timed(ctx, KC_RHS, [&] {
    launch_point_force_rhs(ctx->g, nrhs, ns, ctx->vin.p, ctx->vin.p + nsrc,
                           holes_zero, ctx->vout.p, ldf, ctx->st);
  });
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(f, ctx->vout.p, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

static int matvec_impl(skel_ctx *ctx, int32_t nrhs, const double *x,
                       double *y, int adjoint) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (nrhs < 0 || nrhs > kMaxCols || (nrhs > 0 && (!x || !y)))
    return fail(ctx, SKEL_EINVAL, "invalid matvec arguments");
  if (nrhs == 0) return SKEL_OK;
  const int64_t ldf = nsys(ctx);
  CU(ctx->vin.ensure((size_t)ldf * nrhs));
  CU(ctx->vout.ensure((size_t)ldf * nrhs));
  CU(cudaMemcpyAsync(ctx->vin.p, x, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  // the partial sums take (ranges + 1) x N x 2 doubles per column (2.1 GB
  // at a million nodes): the columns go in batches whose scratch stays
  // within kMatvecScratchBytes (each column's sums do not depend on the
  // batch)
  const size_t per_col = dl_scratch(ctx->N, 1, ctx->N) * sizeof(double);
  const int cb = (int)std::max<size_t>(
      1, std::min<size_t>((size_t)nrhs, kMatvecScratchBytes / per_col));
  CU(ctx->dlscr.ensure(dl_scratch(ctx->N, cb, ctx->N)));
  for (int c0 = 0; c0 < nrhs; c0 += cb) {
    const int nc = std::min(cb, nrhs - c0);
    const double *xin = ctx->vin.p + (int64_t)c0 * ldf;
    double *yout = ctx->vout.p + (int64_t)c0 * ldf;
    timed(ctx, KC_MATVEC, [&] {
      if (ctx->lap)
        launch_lap_matvec(ctx->g, nc, xin, yout, ldf, ctx->dlscr.p, ctx->st);
      else if (adjoint)
        launch_matvec_adjoint(ctx->g, nc, xin, yout, ldf, ctx->dlscr.p,
                              ctx->st);
      else
        launch_matvec(ctx->g, nc, xin, yout, ldf, ctx->dlscr.p, ctx->st);
    });
  }
  ctx->kst[KC_MATVEC].flops += kPairFlops * (double)ctx->N * ctx->N * nrhs;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(y, ctx->vout.p, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

int skel_matvec(skel_ctx *ctx, int32_t nrhs, const double *x, double *y) {
  return matvec_impl(ctx, nrhs, x, y, 0);
}

static int matvec_df_impl(skel_ctx *ctx, int32_t nrhs, const double *x,
                          double *y, int adjoint) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  if (ctx->lap) return stokes_only(ctx);
  if (nrhs < 0 || nrhs > kMaxCols || (nrhs > 0 && (!x || !y)))
    return fail(ctx, SKEL_EINVAL, "invalid matvec arguments");
  if (nrhs == 0) return SKEL_OK;
  const int64_t ldf = nsys(ctx);
  CU(ctx->vin.ensure((size_t)ldf * nrhs));
  CU(ctx->vout.ensure((size_t)ldf * nrhs));
  CU(cudaMemcpyAsync(ctx->vin.p, x, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  int rc;
  for (int q = 0; q < nrhs; ++q)
    if ((rc = op_apply_fast(ctx, ctx->vin.p + (int64_t)q * ldf,
                            ctx->vout.p + (int64_t)q * ldf, adjoint)))
      return rc;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(y, ctx->vout.p, (size_t)ldf * nrhs * sizeof(double),
                     cudaMemcpyDefault, ctx->st));
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  return SKEL_OK;
}

int skel_matvec_df(skel_ctx *ctx, int32_t nrhs, const double *x, double *y) {
  return matvec_df_impl(ctx, nrhs, x, y, 0);
}

int skel_matvec_adjoint_df(skel_ctx *ctx, int32_t nrhs, const double *z,
                           double *y) {
  return matvec_df_impl(ctx, nrhs, z, y, 1);
}

int skel_matvec_adjoint(skel_ctx *ctx, int32_t nrhs, const double *z,
                        double *y) {
  if (ctx && ctx->lap) return stokes_only(ctx);
  return matvec_impl(ctx, nrhs, z, y, 1);
}

int skel_stats(skel_ctx *ctx, char *json, size_t cap) {
  if (!ctx || !json || cap == 0) return SKEL_EINVAL;
  std::ostringstream o;
  o.precision(10);
  o << "{\"N\":" << ctx->N << ",\"p\":" << ctx->p
    << ",\"levels\":" << ctx->tree.L() << ",\"boxes\":" << ctx->tree.boxes.size()
    << ",\"root_skeleton\":" << ctx->s << ",\"t_factor_ms\":" << ctx->t_factor_ms
    << ",\"t_update_ms\":" << ctx->t_update_ms
    << ",\"t_solve_ms\":" << ctx->t_solve_ms
    << ",\"host_factor_ms\":" << ctx->host_factor_ms
    << ",\"alloc_ms\":" << ctx->alloc_ms
    << ",\"cached_device_bytes\":" << dev_cached_bytes()
    << ",\"host_update_ms\":" << ctx->host_update_ms
    << ",\"host_solve_ms\":" << ctx->host_solve_ms
    << ",\"host_prep_ms\":" << ctx->host_prep_ms
    << ",\"host_post_ms\":" << ctx->host_post_ms
    << ",\"last_dirty\":" << ctx->last_dirty
    << ",\"last_boxes\":" << ctx->last_boxes
    << ",\"precision\":\"" << (is_mixed(ctx) ? "mixed" : "fp64") << "\""
    << ",\"id_storage\":\"" << (ctx->id32 ? "fp32" : "fp64") << "\""
    << ",\"factor_storage\":\"" << (ctx->fac32 ? "fp32" : "fp64") << "\""
    << ",\"gmres_iters\":" << ctx->last_iters
    << ",\"gmres_relres\":" << ctx->last_relres
    << ",\"gmres_relres0\":" << ctx->last_relres0
    << ",\"gmres_check\":\"" << (ctx->last_check_df ? "df" : "fp64") << "\""
    << ",\"gmres_recurrence\":" << (ctx->last_check_rec ? 1 : 0)
    << ",\"gmres_fp64_check\":" << (ctx->gmres_fp64_check ? 1 : 0)
    << ",\"flops_factor\":" << ctx->flops_factor
    << ",\"fac_bytes\":" << ctx->fac.used * 8 << ",\"kernels\":{";
  bool first = true;
  for (int c = 0; c < KC_N; ++c) {
    const KStat &k = ctx->kst[c];
    if (k.launches == 0) continue;
    if (!first) o << ",";
    first = false;
    o << "\"" << kKcName[c] << "\":{\"launches\":" << k.launches
      << ",\"ms\":" << k.ms << ",\"flops\":" << k.flops
      << ",\"bytes\":" << k.bytes << "}";
  }
  o << "},\"per_level\":[";
  for (size_t l = 1; l < ctx->lv_nbox.size(); ++l) {
    if (l > 1) o << ",";
    o << "{\"level\":" << l << ",\"boxes\":" << ctx->lv_nbox[l]
      << ",\"max_n\":" << ctx->lv_maxn[l] << ",\"max_k\":" << ctx->lv_maxk[l]
      << ",\"max_m\":" << ctx->lv_maxm[l] << ",\"cluster_boxes\":"
      << ctx->lv_big[l] << ",\"wide_boxes\":" << ctx->lv_wide[l]
      << ",\"moved\":" << ctx->lv_moved[l];
    if (l < ctx->lv_kms.size()) {
      o << ",\"kernel_ms\":{";
      bool f1 = true;
      for (int c = 0; c < KC_N; ++c)
        if (ctx->lv_kms[l][c] > 0) {
          o << (f1 ? "" : ",") << "\"" << kKcName[c]
            << "\":" << ctx->lv_kms[l][c];
          f1 = false;
        }
      o << "}";
    }
    o
      << ",\"ms\":" << ctx->lv_ms[l] << "}";
  }
  o << "]}";
  std::string s = o.str();
  if (s.size() + 1 > cap) return SKEL_ECAPACITY;
  std::memcpy(json, s.c_str(), s.size() + 1);
  return SKEL_OK;
}

int skel_set_tuning(skel_ctx *ctx, const char *key, double value) {
  if (!ctx || !key) return fail(ctx, SKEL_EINVAL, "ctx or key is NULL");
  const std::string k(key);
  const int v = (int)value;
  if (!(value == (double)v))
    return fail(ctx, SKEL_EINVAL, "tuning values are integers");
  if (k == "gmres_fp64_check") {  // a solve setting: the factors stay
    if (v != 0 && v != 1)
      return fail(ctx, SKEL_EINVAL, "gmres_fp64_check is 0 or 1");
    ctx->gmres_fp64_check = v != 0;
    return SKEL_OK;
  }
  if (k == "cluster_min_n" && v >= 1)
    ctx->cluster_min_n = v;
  else if (k == "cluster_level_boxes" && v >= 0)
    ctx->cluster_level_boxes = v;
  else if (k == "sweep_rhs_chunk" && (v == 4 || v == 8 || v == 16))
    ctx->sweep_rhs_chunk = v;
  else if (k == "cluster_mid_min_n" && v >= 1)
    ctx->cluster_mid_min_n = v;
  else if (k == "cluster_mid_level_boxes" && v >= 0)
    ctx->cluster_mid_level_boxes = v;
  else if (k == "wide_min_n" && v >= 1)
    ctx->wide_min_n = v;
  else if (k == "wide_qr_min_n" && v >= 1)
    ctx->wide_qr_min_n = v;
  else if (k == "tc_products" && (v == 0 || v == 1))
    ctx->tc_products = v != 0;
  else
    return fail(ctx, SKEL_EINVAL, "unknown tuning key or invalid value: " + k);
  // the factors were made with the old settings: factor again before use
  drop_graphs(ctx);
  ctx->factored = false;
  return SKEL_OK;
}

int skel_get_tuning(skel_ctx *ctx, const char *key, double *value) {
  if (!ctx || !key || !value) return fail(ctx, SKEL_EINVAL, "NULL argument");
  const std::string k(key);
  if (k == "gmres_fp64_check")
    *value = ctx->gmres_fp64_check ? 1 : 0;
  else if (k == "cluster_min_n")
    *value = ctx->cluster_min_n;
  else if (k == "cluster_level_boxes")
    *value = ctx->cluster_level_boxes;
  else if (k == "sweep_rhs_chunk")
    *value = ctx->sweep_rhs_chunk;
  else if (k == "cluster_mid_min_n")
    *value = ctx->cluster_mid_min_n;
  else if (k == "cluster_mid_level_boxes")
    *value = ctx->cluster_mid_level_boxes;
  else if (k == "wide_min_n")
    *value = ctx->wide_min_n;
  else if (k == "wide_qr_min_n")
    *value = ctx->wide_qr_min_n;
  else if (k == "tc_products")
    *value = ctx->tc_products ? 1 : 0;
  else
    return fail(ctx, SKEL_EINVAL, "unknown tuning key: " + k);
  return SKEL_OK;
}

int skel_set_timing(skel_ctx *ctx, int32_t on) {
  if (!ctx) return fail(nullptr, SKEL_EINVAL, "ctx is NULL");
  CU(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  for (int c = 0; c < KC_N; ++c) ctx->kst[c] = KStat{};
  ctx->timing = on != 0;
  return SKEL_OK;
}

int64_t skel_kernel_launches(void) { return g_launches.load(); }

const char *skel_last_error(skel_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void skel_destroy(skel_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  delete ctx;
}

}  // extern "C"
