"""O-2: straightforward serial recursive skeletonization of the bordered
Stokes system.  Test infrastructure only (see the package docstring).

Follows, in order:
* adaptive quadtree with a fixed root, leaves of at most c nodes (Sec. 2.3);
* per box: the proxy-surface interpolative decomposition (Sec. 2.5,
  Eq. gammaT), one ID for both sides of a nonsymmetric kernel (Sec. 2.4),
  by column-pivoted QR to a relative tolerance (Sec. 2.2);
* elimination of the redundant DOFs by the interpolation matrices of
  Eq. (tmat) and the block elimination of Eq. (schurmat);
* level-by-level compression where every box of a level is compressed from
  the start-of-level state (Sec. 2.7), no compression at the root
  (Eq. bigprods);
* the bordered system of Sec. 3.2 (Eq. bigskel, solution, partition): only
  the top-left block is skeletonized, U H and Psi^T V are carried along and
  the ill-conditioned X_SS is solved inside the top dense block;
* fast updating (Sec. 2.8): boxes whose compression inputs changed are marked
  and only they are refactored, which reproduces a fresh factorization
  exactly when the root is fixed.

Readings where the paper is silent (each listed in the design notes):
* proxy ring: |P| points on the circle of radius proxy_ratio x the box
  half-diagonal, with the double-layer kernel to the ring as target rows and
  Stokeslet plus double-layer sources on the ring as the transposed rows;
* the rank-1 completion N is not a Green's function, so its far part enters
  the ID as two exact rows: (w n)_B and wbar_B n_B (wbar_B = mean weight of
  the box's active nodes);
* skeletons are chosen per DOF; near field F_int = active DOFs of other boxes
  whose node lies strictly inside the proxy disk;
* ID tolerance relative to |R_11|; pivot ties go to the lowest index;
* X_RR conditioning (Sec. 2.2 remark: indices may move from R into S): when
  the partially pivoted LU of X_RR has a pivot at most 1e-3 of its largest,
  Gaussian elimination with diagonal pivoting on X_RR picks the indices
  whose remaining diagonal falls below 1e-3 of the first pivot, those move
  into S with zero rows of T (the ID stays exact), and the box is
  eliminated again once (``xrr_moves``); a pivot ratio that is still below
  1e-14 raises.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .stokes import (Geom, a11_entries, dl_blocks, h_columns, k_entries,
                     psi_columns, quadrature, stokeslet_blocks)


# ---------------------------------------------------------------------------
# tree (Sec. 2.3, Fig. treefig)

@dataclass
class Box:
    key: tuple
    depth: int
    cx: float
    cy: float
    hw: float
    parent: int
    children: list
    nodes: np.ndarray
    is_leaf: bool


@dataclass
class Tree:
    boxes: list
    levels: list
    key2id: dict

    @property
    def L(self):
        return len(self.levels) - 1


def build_tree(x, y, comp, leaf_size) -> Tree:
    """Adaptive quadtree: a fixed root square (the bounding square of
    Gamma_0 with a 1% margin, so it never moves when holes move) is split
    into quadrants until every box holds at most ``leaf_size`` nodes; empty
    boxes are dropped (Sec. 2.3)."""
    x = np.asarray(x)
    y = np.asarray(y)
    outer = np.asarray(comp) == 0
    xmin, xmax = x[outer].min(), x[outer].max()
    ymin, ymax = y[outer].min(), y[outer].max()
    cx, cy = 0.5 * (xmin + xmax), 0.5 * (ymin + ymax)
    hw = 0.5 * max(xmax - xmin, ymax - ymin) * 1.01
    if np.any(np.abs(x - cx) > hw) or np.any(np.abs(y - cy) > hw):
        raise ValueError("node outside the root box")
    boxes, levels, key2id = [], [], {}

    def make(key, depth, bx, by, bh, parent, nodes):
        bid = len(boxes)
        leaf = len(nodes) <= leaf_size
        boxes.append(Box(key, depth, bx, by, bh, parent, [], nodes, leaf))
        key2id[key] = bid
        while len(levels) <= depth:
            levels.append([])
        levels[depth].append(bid)
        if not leaf:
            right = x[nodes] >= bx
            top = y[nodes] >= by
            for q in range(4):
                sel = nodes[(right == bool(q & 1)) & (top == bool(q & 2))]
                if len(sel) == 0:
                    continue
                ccx = bx + 0.5 * bh if q & 1 else bx - 0.5 * bh
                ccy = by + 0.5 * bh if q & 2 else by - 0.5 * bh
                ck = (depth + 1, 2 * key[1] + (q & 1), 2 * key[2] + (q >> 1))
                cid = make(ck, depth + 1, ccx, ccy, 0.5 * bh, bid, sel)
                boxes[bid].children.append(cid)
        return bid

    make((0, 0, 0), 0, cx, cy, hw, -1, np.arange(len(x)))
    return Tree(boxes, levels, key2id)


def proxy_radius(box: Box, ratio):
    return ratio * np.sqrt(2.0) * box.hw


def near_owners(tree: Tree, b: int, level: int, ratio):
    """Boxes other than b that own active DOFs at the start of ``level``
    (boxes of that depth, or leaves above it) and meet b's proxy disk."""
    B = tree.boxes[b]
    rho = proxy_radius(B, ratio)
    out = []
    stack = [0]
    while stack:
        o = stack.pop()
        X = tree.boxes[o]
        dx = max(abs(B.cx - X.cx) - X.hw, 0.0)
        dy = max(abs(B.cy - X.cy) - X.hw, 0.0)
        if dx * dx + dy * dy >= rho * rho:
            continue
        if X.depth == level or X.is_leaf:
            if o != b:
                out.append(o)
        else:
            stack.extend(X.children)
    return sorted(out)


def node_dofs(nodes):
    nodes = np.asarray(nodes, dtype=np.int64)
    return np.stack([2 * nodes, 2 * nodes + 1], axis=1).reshape(-1)


# ---------------------------------------------------------------------------
# interpolative decomposition (Sec. 2.2 and Sec. 2.5, Eq. gammaT)

def cpqr_id(M, tol):
    """Column-pivoted Householder QR of M stopped at the first step whose
    pivot |R_kk| <= tol |R_11|; returns (perm, k, T) with
    M[:, perm[k:]] ~= M[:, perm[:k]] @ T and T = R11^{-1} R12.
    Pivot: largest remaining column norm, ties to the lowest index.  Column
    norms are downdated and recomputed when cancellation makes the downdate
    unreliable (the LAPACK xLAQP2 safeguard)."""
    A = np.array(M, dtype=np.float64, copy=True)
    m, n = A.shape
    perm = np.arange(n)
    if n == 0:
        return perm, 0, np.zeros((0, 0))
    vn1 = np.linalg.norm(A, axis=0)
    vn2 = vn1.copy()
    tol3z = np.sqrt(np.finfo(float).eps)
    k = min(m, n)
    r11 = None
    for j in range(min(m, n)):
        pj = j + int(np.argmax(vn1[j:]))
        if pj != j:
            A[:, [j, pj]] = A[:, [pj, j]]
            perm[[j, pj]] = perm[[pj, j]]
            vn1[[j, pj]] = vn1[[pj, j]]
            vn2[[j, pj]] = vn2[[pj, j]]
        xcol = A[j:, j]
        alpha_abs = np.linalg.norm(xcol)
        if r11 is None:
            r11 = alpha_abs
        if alpha_abs == 0.0 or alpha_abs <= tol * r11:
            k = j
            break
        alpha = -alpha_abs if xcol[0] >= 0 else alpha_abs
        v = xcol.copy()
        v[0] -= alpha
        beta = v @ v
        if j + 1 < n and beta > 0:
            A[j:, j + 1:] -= np.outer(v, (2.0 / beta) * (v @ A[j:, j + 1:]))
        A[j, j] = alpha
        A[j + 1:, j] = 0.0
        for c in range(j + 1, n):
            if vn1[c] == 0.0:
                continue
            t = 1.0 - (abs(A[j, c]) / vn1[c]) ** 2
            t = max(t, 0.0)
            t2 = t * (vn1[c] / vn2[c]) ** 2
            if t2 <= tol3z:
                vn1[c] = np.linalg.norm(A[j + 1:, c])
                vn2[c] = vn1[c]
            else:
                vn1[c] *= np.sqrt(t)
    if k == 0:
        return perm, 0, np.zeros((0, n))
    T = sla.solve_triangular(A[:k, :k], A[:k, k:], lower=False)
    return perm, k, T


def proxy_ring(B: Box, n_proxy, ratio):
    rho = proxy_radius(B, ratio)
    th = 2.0 * np.pi * np.arange(n_proxy) / n_proxy
    px = B.cx + rho * np.cos(th)
    py = B.cy + rho * np.sin(th)
    return px, py, np.cos(th), np.sin(th), np.full(n_proxy,
                                                   2 * np.pi * rho / n_proxy)


def id_matrix(g: Geom, B: Box, act, fint, n_proxy, ratio):
    """Rows whose row space the box's columns must be interpolated in
    (Eq. gammaT with Sec. 2.4): K_{F_int,B}; K_{P,B} (double layer from B to
    the proxy ring); (K_{B,F_int})^T; (G(x_B,P) wbar_B)^T and
    (D(x_B,P) wbar_B)^T (point sources on the ring seen by B); the two rows
    of the far part of the rank-1 completion N.

    The ring sources stand in for the far rows (K_{B,F})^T, whose entries
    carry the far nodes' quadrature weights, so they are weighted by the
    box's mean node weight wbar_B rather than by the ring's own quadrature
    weight 2 pi rho / P: the relative ID tolerance then means the same for
    them as for the near-field and target-side rows at every level and
    every discretization size."""
    nodes = act // 2
    comp = act % 2
    ii = np.arange(len(act))
    px, py, pnx, pny, pw = proxy_ring(B, n_proxy, ratio)
    rows = [k_entries(g, fint, act)]
    D = dl_blocks(px, py, g.x[nodes], g.y[nodes], g.nx[nodes], g.ny[nodes],
                  g.w[nodes])                                # (P, n, 2, 2)
    rows.append(np.concatenate([D[:, ii, 0, comp], D[:, ii, 1, comp]], 0))
    rows.append(k_entries(g, act, fint).T)
    wbar = np.mean(g.w[nodes]) if len(nodes) else 0.0
    G = stokeslet_blocks(g.x[nodes], g.y[nodes], px, py) * wbar
    rows.append(np.concatenate([G[ii, :, comp, 0].T, G[ii, :, comp, 1].T], 0))
    Ds = dl_blocks(g.x[nodes], g.y[nodes], px, py, pnx, pny,
                   np.full(n_proxy, wbar))
    rows.append(np.concatenate([Ds[ii, :, comp, 0].T, Ds[ii, :, comp, 1].T],
                               0))
    nvec = np.where(comp == 0, g.nx[nodes], g.ny[nodes])
    rows.append((g.w[nodes] * nvec)[None, :])
    rows.append((wbar * nvec)[None, :])
    return np.concatenate(rows, axis=0)


# ---------------------------------------------------------------------------
# factorization

@dataclass
class BoxRecord:
    act: np.ndarray       # active DOFs at the start of the box's level
    perm: np.ndarray
    k: int
    skel: np.ndarray
    red: np.ndarray
    T: np.ndarray         # k x r
    lu: tuple             # LU of X_RR (lu, piv)
    Y: np.ndarray         # X_RR^{-1} X_RS   (r x k)
    Z: np.ndarray         # X_SR X_RR^{-1}   (k x r)
    XSS: np.ndarray       # K_SS - X_SR X_RR^{-1} X_RS  (k x k)
    near: list = field(default_factory=list)


@dataclass
class Factorization:
    g: Geom
    tree: Tree
    params: dict
    rec: dict             # box id -> BoxRecord
    content: dict         # box id -> subtree content digest
    root_act: np.ndarray
    A_root: np.ndarray
    UH: np.ndarray        # U H before the X_RR solves (2N x 3p)
    W: np.ndarray         # X_RR^{-1} (U H)_R on R rows, U H on root rows
    QT: np.ndarray        # V^T Psi before the X_RR^{-T} solves
    Wt: np.ndarray        # X_RR^{-T} (V^T Psi)_R on R rows
    G: np.ndarray         # (Psi^T V)_R X_RR^{-1} (U H)_R  (3p x 3p)
    top: np.ndarray
    top_lu: tuple
    rmask: np.ndarray     # True on every DOF eliminated below the root
    dirty: dict = field(default_factory=dict)


def _content_digest(g: Geom, nodes):
    h = hashlib.sha1()
    for arr in (np.asarray(nodes, np.int64), g.x[nodes], g.y[nodes],
                g.nx[nodes], g.ny[nodes], g.w[nodes], g.kap[nodes]):
        h.update(np.ascontiguousarray(arr).tobytes())
    return h.hexdigest()


def _diag_block(g: Geom, tree: Tree, b, act, rec):
    """Start-of-level diagonal block of box b: for a leaf, entries of
    -1/2 I + D + N; above the leaves, the children's Schur complements X_SS
    on the diagonal and original entries between siblings (Eq. levelcompress)."""
    A = a11_entries(g, act, act)
    off = 0
    for c in tree.boxes[b].children:
        kc = rec[c].k
        A[off:off + kc, off:off + kc] = rec[c].XSS
        off += kc
    return A


# X_RR conditioning (Sec. 2.2 remark).  The operator's null space (rigid
# motions of every hole that lies wholly inside a box) makes X_RR of such
# boxes nearly singular.  When the partially pivoted LU of X_RR has a pivot
# at most MOVE_RATIO of its largest, Gaussian elimination with diagonal
# pivoting on X_RR finds the indices to keep: it stops once the largest
# remaining diagonal entry is at most MOVE_RATIO of the first pivot, and
# the indices not eliminated by then move from R into S.
MOVE_RATIO = 1e-3


def xrr_moves(XRR, ratio=MOVE_RATIO):
    """Positions in R to move into S (ascending): the indices left over by
    elimination with diagonal (symmetric) pivoting on X_RR, stopped when the
    largest remaining |diagonal| is at most ratio times the first pivot, so
    the principal block on the eliminated indices is well conditioned."""
    A = np.array(XRR, dtype=np.float64, copy=True)
    r = A.shape[0]
    left = np.ones(r, dtype=bool)
    first = None
    for _ in range(r):
        cand = np.where(left)[0]
        p = cand[int(np.argmax(np.abs(np.diag(A)[cand])))]
        a = A[p, p]
        if first is None:
            first = abs(a)
        if not abs(a) > ratio * first:
            break
        left[p] = False
        rest = np.where(left)[0]
        A[np.ix_(rest, rest)] -= np.outer(A[rest, p], A[p, rest]) / a
    return np.where(left)[0] if first is not None else np.zeros(0, int)


def _compress(g: Geom, tree: Tree, b, act, fint, A, params, near):
    """Compress one box: ID (Sec. 2.5), then Eq. (tmat) and Eq. (schurmat),
    moving indices from R into S while X_RR is ill-conditioned."""
    B = tree.boxes[b]
    M = id_matrix(g, B, act, fint, params["n_proxy"], params["proxy_ratio"])
    perm, k, T = cpqr_id(M, params["id_tol"])
    for attempt in range(2):
        K = A[np.ix_(perm, perm)]
        KSS, KSR = K[:k, :k], K[:k, k:]
        KRS, KRR = K[k:, :k], K[k:, k:]
        XRS = KRS - T.T @ KSS
        XSR = KSR - KSS @ T
        XRR = KRR - T.T @ KSR - XRS @ T
        r = len(act) - k
        if r == 0:
            break
        lu = sla.lu_factor(XRR, check_finite=True)
        d = np.abs(np.diag(lu[0]))
        if attempt == 1 or d.min() > MOVE_RATIO * d.max():
            break
        # S' = S + J, R' = R - J; T' = [T restricted to R'; 0] keeps
        # K_{F,R'} ~ K_{F,S'} T' and makes X_{R'R'} a principal block of X_RR
        J = xrr_moves(XRR)
        if len(J) == 0:
            break
        keep = np.setdiff1d(np.arange(r), J)
        perm = np.concatenate([perm[:k], perm[k:][J], perm[k:][keep]])
        T = np.vstack([T[:, keep], np.zeros((len(J), len(keep)))])
        k += len(J)
    r = len(act) - k
    if r > 0:
        if d.min() <= 1e-14 * d.max():
            raise FloatingPointError(f"X_RR of box {B.key} is singular")
        Y = sla.lu_solve(lu, XRS)
        Z = sla.lu_solve(lu, XSR.T, trans=1).T
    else:
        lu = (np.zeros((0, 0)), np.zeros(0, dtype=np.int32))
        Y = np.zeros((0, k))
        Z = np.zeros((k, 0))
    XSS = KSS - XSR @ Y
    return BoxRecord(act=act, perm=perm, k=k, skel=act[perm[:k]],
                     red=act[perm[k:]], T=T, lu=lu, Y=Y, Z=Z, XSS=XSS,
                     near=near)


def _level_act(tree: Tree, b, rec):
    B = tree.boxes[b]
    if B.is_leaf:
        return node_dofs(B.nodes)
    return np.concatenate([rec[c].skel for c in B.children]).astype(np.int64)


def _owner_act(tree, o, level, act_of):
    X = tree.boxes[o]
    if X.depth == level:
        return act_of[o]
    return node_dofs(X.nodes)        # a leaf above this level: all its DOFs


def factor(wl, params=None, old: Factorization | None = None,
           g: Geom | None = None) -> Factorization:
    """Recursive skeletonization of -1/2 I + D + N level by level (Sec. 2.3,
    Sec. 2.7), then the bordered top block of Sec. 3.2.  With ``old`` given,
    this is the fast update of Sec. 2.8: only boxes whose compression inputs
    changed are recompressed and every other record is reused."""
    if params is None:
        params = dict(leaf_size=wl.leaf_size, n_proxy=wl.n_proxy,
                      proxy_ratio=wl.proxy_ratio, id_tol=wl.id_tol)
    if g is None:
        g = quadrature(wl)
    tree = build_tree(g.x, g.y, g.comp, params["leaf_size"])
    ratio = params["proxy_ratio"]
    content = {b: _content_digest(g, B.nodes) for b, B in
               enumerate(tree.boxes)}
    rec, dirty = {}, {}
    for level in range(tree.L, 0, -1):
        act_of = {b: _level_act(tree, b, rec) for b in tree.levels[level]}
        changed = {}
        if old is not None:
            changed = _changed_owners(tree, old, content, level, dirty)
        for b in tree.levels[level]:
            B = tree.boxes[b]
            near = near_owners(tree, b, level, ratio)
            if old is not None:
                ob = old.tree.key2id.get(B.key)
                near_keys = [tree.boxes[o].key for o in near]
                old_near = None if ob is None else \
                    [old.tree.boxes[o].key for o in old.rec[ob].near]
                dirty[b] = (changed[b] or any(changed[o] for o in near)
                            or near_keys != old_near)
                if not dirty[b]:
                    r0 = old.rec[ob]
                    rec[b] = BoxRecord(**{**r0.__dict__, "near": near})
                    continue
            rho = proxy_radius(B, ratio)
            fint = []
            for o in near:
                d = _owner_act(tree, o, level, act_of)
                n = d // 2
                inside = (g.x[n] - B.cx) ** 2 + (g.y[n] - B.cy) ** 2 < rho ** 2
                fint.append(d[inside])
            fint = np.concatenate(fint) if fint else np.zeros(0, np.int64)
            act = act_of[b]
            A = _diag_block(g, tree, b, act, rec)
            rec[b] = _compress(g, tree, b, act, fint, A, params, near)
    root = tree.boxes[0]
    root_act = node_dofs(root.nodes) if root.is_leaf else \
        np.concatenate([rec[c].skel for c in root.children]).astype(np.int64)
    A_root = _diag_block(g, tree, 0, root_act, rec) if not root.is_leaf \
        else a11_entries(g, root_act, root_act)
    fac = Factorization(g=g, tree=tree, params=params, rec=rec,
                        content=content, root_act=root_act, A_root=A_root,
                        UH=None, W=None, QT=None, Wt=None, G=None, top=None,
                        top_lu=None, rmask=None, dirty=dirty)
    _bordered(fac)
    return fac


def _changed_owners(tree, old, content, level, dirty):
    """in_changed for every owner at the start of ``level``: the box is new,
    its subtree content (node ids and geometry) differs, its leaf status
    differs, or one of its children was refactored."""
    out = {}
    for o, X in enumerate(tree.boxes):
        if not (X.depth == level or (X.is_leaf and X.depth < level)):
            continue
        ob = old.tree.key2id.get(X.key)
        if ob is None:
            out[o] = True
            continue
        OX = old.tree.boxes[ob]
        ch = (old.content[ob] != content[o]) or (OX.is_leaf != X.is_leaf)
        if X.depth == level and not X.is_leaf:
            ch = ch or any(dirty[c] for c in X.children)
        out[o] = ch
    return out


def update(old: Factorization, wl_new) -> Factorization:
    """Fast update after moved nodes (Sec. 2.8); exact w.r.t. a fresh
    factorization because the root is fixed and the tree is a pure function
    of the node set."""
    return factor(wl_new, old.params, old=old)


# ---------------------------------------------------------------------------
# apply / solve (Eq. kinv, Sec. 2.7 last paragraph, Sec. 3.2)

def _levels_up(fac):
    for level in range(fac.tree.L, 0, -1):
        for b in fac.tree.levels[level]:
            yield fac.rec[b]


def _levels_down(fac):
    for level in range(1, fac.tree.L + 1):
        for b in fac.tree.levels[level]:
            yield fac.rec[b]


def _up_sweep(fac, b, adjoint=False, pre=None):
    """Apply U (box by box: L_T then G_L, Eq. tmat/schurmat) or, with
    ``adjoint``, V^T (R_T^T then G_R^T), solving each X_RR (X_RR^T) right
    after its box.  ``pre`` receives the R rows before the solve."""
    for r in _levels_up(fac):
        S, R = r.skel, r.red
        if len(R) == 0:
            continue
        b[R] -= r.T.T @ b[S]
        b[S] -= (r.Y.T if adjoint else r.Z) @ b[R]
        if pre is not None:
            pre[R] = b[R]
        b[R] = sla.lu_solve(r.lu, b[R], trans=1 if adjoint else 0)
    return b


def _down_sweep(fac, y, adjoint=False):
    """Apply V (G_R then R_T) or, with ``adjoint``, U^T (G_L^T then L_T^T),
    top level first."""
    for r in _levels_down(fac):
        S, R = r.skel, r.red
        if len(R) == 0:
            continue
        y[R] -= (r.Z.T if adjoint else r.Y) @ y[S]
        y[S] -= r.T @ y[R]
    return y


def _bordered(fac):
    """Carry H and Psi through the factors (Eq. bigskel) and form the top
    dense block of Eq. (partition):
    [[X_SS, (UH)_S], [(Psi^T V)_S, -I - (Psi^T V)_R X_RR^{-1} (UH)_R]]."""
    g = fac.g
    n2 = 2 * g.N
    p3 = 3 * g.p
    dofs = np.arange(n2)
    rmask = np.ones(n2, dtype=bool)
    rmask[fac.root_act] = False
    UH = np.zeros((n2, p3))
    W = h_columns(g, dofs)
    _up_sweep(fac, W, adjoint=False, pre=UH)
    UH[~rmask] = W[~rmask]
    QT = np.zeros((n2, p3))
    Wt = psi_columns(g, dofs)
    _up_sweep(fac, Wt, adjoint=True, pre=QT)
    QT[~rmask] = Wt[~rmask]
    G = QT[rmask].T @ W[rmask]
    s = len(fac.root_act)
    top = np.zeros((s + p3, s + p3))
    top[:s, :s] = fac.A_root
    top[:s, s:] = UH[fac.root_act]
    top[s:, :s] = QT[fac.root_act].T
    top[s:, s:] = -np.eye(p3) - G
    fac.UH, fac.W, fac.QT, fac.Wt, fac.G = UH, W, QT, Wt, G
    fac.top = top
    fac.top_lu = sla.lu_factor(top)
    fac.rmask = rmask


def solve(fac: Factorization, f, adjoint=False):
    """[mu; lambda] from [f; g] through the factorization: up-sweep b = U f
    with the X_RR solves, the top dense block of Eq. (partition), the R
    unknowns by back substitution, then the down-sweep mu = V y
    (Eq. solution).  ``adjoint`` solves with the transposed system."""
    g = fac.g
    n2 = 2 * g.N
    f = np.asarray(f, dtype=np.float64)
    one = f.ndim == 1
    if one:
        f = f[:, None]
    b = f[:n2].copy()
    gl = f[n2:]
    _up_sweep(fac, b, adjoint=adjoint)
    rm = fac.rmask
    S = fac.root_act
    couple = fac.UH if adjoint else fac.QT
    rhs = np.concatenate([b[S], gl - couple[rm].T @ b[rm]], axis=0)
    top = sla.lu_solve(fac.top_lu, rhs, trans=1 if adjoint else 0)
    s = len(S)
    lam = top[s:]
    y = b
    y[rm] -= (fac.Wt if adjoint else fac.W)[rm] @ lam
    y[S] = top[:s]
    _down_sweep(fac, y, adjoint=adjoint)
    out = np.concatenate([y, lam], axis=0)
    return out[:, 0] if one else out


def solve_adjoint(fac: Factorization, f):
    return solve(fac, f, adjoint=True)
