// Host quadtree for the skeletonization (Sec. 2.3, Fig. treefig): a fixed
// root square split into quadrants until every box holds at most leaf_size
// nodes; empty boxes are dropped.  The tree is a pure function of the node
// positions and the root, which is what makes updating exact (Sec. 2.8).
#include <algorithm>
#include <cmath>

#include "skel_internal.h"

namespace skel {

static int make_box(Tree &t, const double *x, const double *y, int depth,
                    int64_t ix, int64_t iy, double cx, double cy, double hw,
                    int parent, int64_t nbeg, int64_t ncnt, int leaf_size,
                    std::vector<int64_t> &tmp) {
  int id = (int)t.boxes.size();
  HBox B;
  B.depth = depth;
  B.ix = ix;
  B.iy = iy;
  B.cx = cx;
  B.cy = cy;
  B.hw = hw;
  B.parent = parent;
  B.nchild = 0;
  for (int q = 0; q < 4; ++q) B.child[q] = -1;
  B.nbeg = nbeg;
  B.ncnt = ncnt;
  B.leaf = ncnt <= leaf_size;
  t.boxes.push_back(B);
  t.key2id[box_key(depth, ix, iy)] = id;
  if ((int)t.levels.size() <= depth) t.levels.resize(depth + 1);
  t.levels[depth].push_back(id);
  if (B.leaf) return id;
  // stable partition of the (ascending) node range into quadrants
  // q = (x >= cx) + 2 (y >= cy)
  int64_t cnt[4] = {0, 0, 0, 0};
  for (int64_t i = nbeg; i < nbeg + ncnt; ++i) {
    int64_t j = t.order[i];
    int q = (x[j] >= cx ? 1 : 0) + (y[j] >= cy ? 2 : 0);
    cnt[q]++;
  }
  int64_t start[4];
  start[0] = 0;
  for (int q = 1; q < 4; ++q) start[q] = start[q - 1] + cnt[q - 1];
  tmp.resize(ncnt);
  int64_t fill[4] = {start[0], start[1], start[2], start[3]};
  for (int64_t i = nbeg; i < nbeg + ncnt; ++i) {
    int64_t j = t.order[i];
    int q = (x[j] >= cx ? 1 : 0) + (y[j] >= cy ? 2 : 0);
    tmp[fill[q]++] = j;
  }
  std::copy(tmp.begin(), tmp.begin() + ncnt, t.order.begin() + nbeg);
  for (int q = 0; q < 4; ++q) {
    if (cnt[q] == 0) continue;
    double ccx = (q & 1) ? cx + 0.5 * hw : cx - 0.5 * hw;
    double ccy = (q & 2) ? cy + 0.5 * hw : cy - 0.5 * hw;
    int cid = make_box(t, x, y, depth + 1, 2 * ix + (q & 1), 2 * iy + (q >> 1),
                       ccx, ccy, 0.5 * hw, id, nbeg + start[q], cnt[q],
                       leaf_size, tmp);
    HBox &P = t.boxes[id];
    P.child[P.nchild++] = cid;
  }
  return id;
}

void build_tree_root(const double *x, const double *y, int64_t N,
                     int leaf_size, double cx, double cy, double hw, Tree &t) {
  t.boxes.clear();
  t.levels.clear();
  t.key2id.clear();
  t.order.resize(N);
  for (int64_t i = 0; i < N; ++i) t.order[i] = i;
  std::vector<int64_t> tmp;
  make_box(t, x, y, 0, 0, 0, cx, cy, hw, -1, 0, N, leaf_size, tmp);
}

bool build_tree(const double *x, const double *y, const int32_t *comp,
                int64_t N, int leaf_size, Tree &t, std::string &err) {
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  int64_t n0 = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (comp[i] != 0) continue;
    ++n0;
    xmin = std::min(xmin, x[i]);
    xmax = std::max(xmax, x[i]);
    ymin = std::min(ymin, y[i]);
    ymax = std::max(ymax, y[i]);
  }
  if (n0 == 0) {
    err = "no node on the outer curve (comp == 0)";
    return false;
  }
  double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
  double hw = 0.5 * std::max(xmax - xmin, ymax - ymin) * 1.01;
  for (int64_t i = 0; i < N; ++i) {
    if (!(std::fabs(x[i] - cx) <= hw && std::fabs(y[i] - cy) <= hw)) {
      err = "node " + std::to_string(i) + " lies outside the root box";
      return false;
    }
  }
  build_tree_root(x, y, N, leaf_size, cx, cy, hw, t);
  return true;
}

void near_owners(const Tree &t, int b, int level, double ratio,
                 std::vector<int> &out) {
  out.clear();
  const HBox &B = t.boxes[b];
  double rho = proxy_radius(B, ratio);
  thread_local std::vector<int> stack;  // reused across calls
  stack.assign(1, 0);
  while (!stack.empty()) {
    int o = stack.back();
    stack.pop_back();
    const HBox &X = t.boxes[o];
    double dx = std::max(std::fabs(B.cx - X.cx) - X.hw, 0.0);
    double dy = std::max(std::fabs(B.cy - X.cy) - X.hw, 0.0);
    if (dx * dx + dy * dy >= rho * rho) continue;
    if (X.depth == level || X.leaf) {
      if (o != b) out.push_back(o);
    } else {
      for (int c = 0; c < X.nchild; ++c) stack.push_back(X.child[c]);
    }
  }
  std::sort(out.begin(), out.end());
}

}  // namespace skel
