"""Element-wise parity on the paths that only large boxes take.

* The 64 clustered holes of the quadrant workload with 32 nodes per hole
  and 2048 on the outer circle (4096 nodes, leaves of 128): boxes hold
  whole holes, so the LU of X_RR finds tiny pivots and indices move from R
  into S (Sec. 2.2 remark, Sec. 3.2), and the largest boxes run on the
  16-CTA cluster kernels.  The full solution and the adjoint solution,
  every entry, against the dense LU of the exact bordered system, in the
  FP64 and in the mixed form.  This system has condition number 2.1e6, so
  the forward error of any solver at backward error 1e-12 can reach 2e-6;
  the oracle's own skeletonization (ID tolerance 1e-12) realises 1.3e-9 on
  mu and 3e-11 on lambda.  The forward check is therefore 1e-8 here, and
  the normwise backward error (the largest residual row against the dense
  matrix, relative to ||A|| max|x| + max|b|) must meet the 1e-10 target.
* The 16-hole star at half its node counts (16384 nodes): the GPU solution
  against the oracle's own skeletonization (same readings, independent
  code), every entry, and both against the exact point-force velocity.

Per block: mu against max|mu|, lambda against its scale
(gpu_util.block_errors)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_solution_close, assert_velocity_close, solver

pytestmark = pytest.mark.gpu

TOL = 1e-10


def quad_holes32():
    """The quadrant workload's curves, 2048 nodes on the outer circle and
    32 on each of the 64 holes, leaves of 128 nodes."""
    from workloads.configs import _flatten
    q = W.quad64()
    return _flatten("quad64-h32", q.curves, [2048] + [32] * 64,
                    src_xy=q.src_xy[:2], src_f=q.src_f[:2],
                    rhs_holes_zero=False, targets=q.targets[:64],
                    leaf_size=128)


@pytest.fixture(scope="module")
def quad32():
    import scipy.linalg as sla
    wl = quad_holes32()
    g = oracle.quadrature(wl)
    A = oracle.dense_system(g)
    f = oracle.boundary_data(g, wl.src_xy[:2], wl.src_f[:2])
    rng = np.random.default_rng(31)
    rhs = np.concatenate([f, rng.standard_normal((A.shape[0], 2))], axis=1)
    lu = sla.lu_factor(A)
    x = sla.lu_solve(lu, rhs)
    xt = sla.lu_solve(lu, rhs, trans=1)
    return wl, A, rhs, x, xt


def backward_error(A, x, b):
    """Normwise backward error per column, the largest over the columns:
    max_i |A x - b|_i / (||A||_inf max|x| + max|b|)."""
    x = np.asarray(x).reshape(A.shape[0], -1)
    b = np.asarray(b).reshape(A.shape[0], -1)
    na = np.abs(A).sum(axis=1).max()
    r = np.abs(A @ x - b).max(axis=0)
    return float((r / (na * np.abs(x).max(axis=0) +
                       np.abs(b).max(axis=0))).max())


def _mixed(wl):
    import paper_2001_11619_gb300 as skel
    return solver(wl, precision=skel.MIXED, id_tol=1e-6, gmres_tol=1e-12,
                  gmres_maxit=80)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_quad_holes_whole_holes_element_wise(quad32, form):
    wl, A, rhs, x, xt = quad32
    s = _mixed(wl) if form == "mixed" else solver(wl)
    s.factor()
    st = s.stats()
    if form == "fp64":
        # the X_RR split ran, and the largest boxes went to the clusters
        assert sum(lv["moved"] for lv in st["per_level"]) > 0
    assert sum(lv["cluster_boxes"] for lv in st["per_level"]) > 0
    xs = np.asarray(s.solve(rhs))
    assert backward_error(A, xs, rhs) < TOL
    assert_solution_close(xs, x, wl, 1e-8, f"{form} solve")
    zs = np.asarray(s.solve_adjoint(rhs))
    assert backward_error(A.T, zs, rhs) < TOL
    assert_solution_close(zs, xt, wl, 1e-8, f"{form} adjoint")
    tx, ty = wl.targets[:, 0].copy(), wl.targets[:, 1].copy()
    u = s.eval_velocity(xs[:, :2], tx, ty)
    for c in range(2):
        ue = oracle.point_force_velocity(tx, ty, wl.src_xy[c], wl.src_f[c])
        assert_velocity_close(u[:, :, c], ue, TOL, f"{form} velocity {c}")
    s.close()


def test_star16_half_against_oracle_skeletonization():
    wl = W.scaled(W.star16(), 2, n_targets=128)
    assert wl.N == 16384
    g = oracle.quadrature(wl)
    f = oracle.boundary_data(g, wl.src_xy, wl.src_f)
    fac = oracle.factor(wl)
    xo = oracle.solve(fac, f)
    s = solver(wl)
    s.factor()
    st = s.stats()
    assert st["levels"] == fac.tree.L
    assert st["boxes"] == len(fac.tree.boxes)
    xs = s.solve(f)
    assert_solution_close(xs, xo, wl, TOL, "GPU vs oracle skeletonization")
    tx, ty = wl.targets[:, 0].copy(), wl.targets[:, 1].copy()
    ue = oracle.point_force_velocity(tx, ty, wl.src_xy[0], wl.src_f[0])
    assert_velocity_close(s.eval_velocity(xs, tx, ty)[:, :, 0], ue, TOL,
                          "GPU velocity")
    assert_velocity_close(oracle.interior_velocity(g, xo, tx, ty)[:, :, 0],
                          ue, TOL, "oracle velocity")
    s.close()


def test_wide_elimination_against_cluster_path_and_dense(quad32):
    """Boxes of at least wide_min_n active DOFs are eliminated by launches
    over the whole GPU (tiled GEMMs, blocked LU of X_RR, blocked triangular
    solves), and of at least wide_qr_min_n also run their column-pivoted QR
    that way.  With the threshold low enough that most cluster-class boxes
    take that path, the solution matches the all-cluster factorization to
    rounding, and both meet the dense checks; the X_RR moves happen on the
    wide path too."""
    wl, A, rhs, x, xt = quad32
    a = solver(wl)
    a.set_tuning(wide_min_n=1 << 30, wide_qr_min_n=1 << 30)   # all clusters
    a.factor()
    assert all(lv["wide_boxes"] == 0 for lv in a.stats()["per_level"])
    b = solver(wl)
    b.set_tuning(wide_min_n=200, wide_qr_min_n=200)
    b.factor()
    st = b.stats()
    assert sum(lv["wide_boxes"] for lv in st["per_level"]) > 0
    assert sum(lv["moved"] for lv in st["per_level"]) > 0
    # the CPQR of the wide boxes sums in another order: rank decisions near
    # the tolerance may differ by a few indices
    ka, kb = a.stats()["root_skeleton"], st["root_skeleton"]
    assert abs(ka - kb) <= 0.02 * ka + 2
    xa, xb = np.asarray(a.solve(rhs)), np.asarray(b.solve(rhs))
    assert_solution_close(xb, xa, wl, 1e-9, "wide vs cluster")
    for xs in (xa, xb):
        assert backward_error(A, xs, rhs) < TOL
        assert_solution_close(xs, x, wl, 1e-8)
    zb = np.asarray(b.solve_adjoint(rhs))
    assert backward_error(A.T, zb, rhs) < TOL
    assert_solution_close(zb, xt, wl, 1e-8, "wide adjoint")
    a.close()
    b.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_wide_update_equals_fresh_bitwise(form):
    """A moved hole on the clustered-hole geometry with the wide path on:
    the update recompresses the top boxes through it and equals a fresh
    factorization bit for bit (Sec. 2.8), solve and adjoint solve."""
    from gpu_util import to_device
    wl = quad_holes32()
    mk = _mixed if form == "mixed" else solver
    s = mk(wl)
    s.set_tuning(wide_min_n=200, wide_qr_min_n=200)
    s.factor()
    h, d = W.random_moves(wl, 1, seed=11)[0]
    moved = W.move_hole(wl, h, d)
    sl = moved.node_slice(h)
    s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(moved))
    assert 0 < s.stats()["last_dirty"] < s.stats()["last_boxes"]
    fresh = mk(moved)
    fresh.set_tuning(wide_min_n=200, wide_qr_min_n=200)
    fresh.factor()
    assert sum(lv["wide_boxes"] for lv in fresh.stats()["per_level"]) > 0
    rhs = np.random.default_rng(3).standard_normal((wl.n_unknowns, 2))
    assert np.array_equal(np.asarray(s.solve(rhs)),
                          np.asarray(fresh.solve(rhs)))
    assert np.array_equal(np.asarray(s.solve_adjoint(rhs)),
                          np.asarray(fresh.solve_adjoint(rhs)))
    s.close()
    fresh.close()
