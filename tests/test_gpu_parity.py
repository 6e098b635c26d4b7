"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: 1e-10 relative on the solution [mu; lambda] and on interior
velocities, the accuracy target of the FP64 form at ID tolerance 1e-12.
Building blocks with no approximation (boundary data, operator apply,
velocity evaluation) must match to rounding (1e-13)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import (assert_solution_close, assert_velocity_close, rel,
                      solver)

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def c1():
    wl = W.star1()
    g = oracle.quadrature(wl)
    f = oracle.boundary_data(g, wl.src_xy, wl.src_f)
    A = oracle.dense_system(g)
    return wl, g, f, A, np.linalg.solve(A, f)


@pytest.fixture(scope="module")
def c1_solver(c1):
    wl = c1[0]
    s = solver(wl)
    s.factor()
    return s


def test_boundary_data_matches(c1, c1_solver):
    wl, g, f, A, x = c1
    fg = c1_solver.point_force_rhs(wl.src_xy, wl.src_f)
    assert rel(fg, f) < 1e-13


def test_operator_apply_matches(c1, c1_solver):
    wl, g, f, A, x = c1
    rng = np.random.default_rng(1)
    v = rng.standard_normal((A.shape[0], 2))
    assert rel(c1_solver.matvec(v), A @ v) < 1e-13


def test_solve_matches_dense_oracle(c1, c1_solver):
    wl, g, f, A, x = c1
    xs = c1_solver.solve(f)
    assert_solution_close(xs, x, wl, TOL)


def test_adjoint_operator_apply_matches(c1, c1_solver):
    wl, g, f, A, x = c1
    rng = np.random.default_rng(5)
    v = rng.standard_normal((A.shape[0], 2))
    assert rel(c1_solver.matvec_adjoint(v), A.T @ v) < 1e-13


def test_double_float_operator_apply(c1, c1_solver):
    """The double-float operator of the GMRES iterations and its transpose:
    within 2e-13 of the dense FP64 matrix (and of the FP64 apply)."""
    wl, g, f, A, x = c1
    rng = np.random.default_rng(12)
    v = rng.standard_normal((A.shape[0], 2))
    y = c1_solver.matvec_df(v)
    assert rel(y, A @ v) < 2e-13
    assert rel(y, c1_solver.matvec(v)) < 2e-13
    # and its transpose (the products of the mixed adjoint solve)
    yt = c1_solver.matvec_adjoint_df(v)
    assert rel(yt, A.T @ v) < 2e-13
    # a smooth density (the solution) too
    assert rel(c1_solver.matvec_df(x), A @ x) < 2e-13


def _mixed(wl, **kw):
    import paper_2001_11619_gb300 as skel
    kw.setdefault("id_tol", 1e-6)
    kw.setdefault("gmres_tol", 1e-13)
    kw.setdefault("gmres_maxit", 60)
    return solver(wl, precision=skel.MIXED, **kw)


def test_mixed_form_reaches_fp64_accuracy(c1):
    """FP32 factors (FP64 rank decisions, T solves and top block) as the
    preconditioner of GMRES on the FP64 operator: same 1e-10 target."""
    wl, g, f, A, x = c1
    s = _mixed(wl)
    s.factor()
    xs = s.solve(f)
    st = s.stats()
    assert st["precision"] == "mixed"
    assert st["id_storage"] == "fp32"
    assert st["factor_storage"] == "fp64"
    assert st["gmres_relres"] <= 1e-13
    # the FP32 factorization at id_tol 1e-6 is a preconditioner of about
    # that quality: GMRES needs few iterations
    assert st["gmres_relres0"] < 2e-5
    assert 0 < st["gmres_iters"] <= 4
    assert_solution_close(xs, x, wl, TOL)
    rng = np.random.default_rng(6)
    rhs = rng.standard_normal((A.shape[0], 2))
    assert_solution_close(s.solve_adjoint(rhs), np.linalg.solve(A.T, rhs),
                          wl, TOL, "adjoint")
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    u = s.eval_velocity(xs, tx, ty)[:, :, 0]
    ue = oracle.point_force_velocity(tx, ty, wl.src_xy[0], wl.src_f[0])
    assert_velocity_close(u, ue, TOL)


def test_graph_replayed_solves_equal_direct_solves(c1):
    """One-column solves are replayed from a CUDA graph captured on the
    first of them (the GMRES preconditioner and single solves, both
    directions).  The replays give the same bits as the direct launches
    (per-kernel timing on, which turns the graphs off), and an update
    recaptures them."""
    import paper_2001_11619_gb300 as skel
    wl, g, f, A, x = c1
    for prec in (skel.FP64, skel.MIXED):
        s = _mixed(wl) if prec == skel.MIXED else solver(wl)
        s.factor()
        first = s.solve(f)
        l0 = skel.kernel_launches()
        replay = s.solve(f)
        adj = [s.solve_adjoint(f), s.solve_adjoint(f)]
        assert skel.kernel_launches() > l0  # replays are counted
        s.set_timing(True)
        direct = s.solve(f)
        adj_direct = s.solve_adjoint(f)
        s.set_timing(False)
        assert np.array_equal(first, replay)
        assert np.array_equal(replay, direct)
        assert np.array_equal(adj[0], adj[1])
        assert np.array_equal(adj[1], adj_direct)
        assert_solution_close(replay, x, wl, TOL)
        moved = W.move_hole(wl, 1, (0.01, 0.004))
        ids = np.arange(wl.node_slice(1).start, wl.node_slice(1).stop)
        from gpu_util import to_device
        s.update_moved_nodes(ids, to_device(moved))
        f2 = oracle.boundary_data(oracle.quadrature(moved), wl.src_xy,
                                  wl.src_f)
        a, b = s.solve(f2), s.solve(f2)
        s.set_timing(True)
        c = s.solve(f2)
        assert np.array_equal(a, b) and np.array_equal(b, c)
        x2 = np.linalg.solve(oracle.dense_system(oracle.quadrature(moved)),
                             f2)
        assert_solution_close(b, x2, wl, TOL)
        s.close()


def test_mixed_ranks_track_fp64_ranks(c1):
    """FP32 storage must not change the rank decisions materially: at the
    same ID tolerance the skeleton sizes of the FP32 and the FP64
    factorizations agree to a few percent (drifting pivot norms in FP32
    would stop the CPQR early and shrink them)."""
    wl = c1[0]
    a = _mixed(wl)
    a.factor()
    b = solver(wl, id_tol=1e-6)
    b.factor()
    ka, kb = a.stats()["root_skeleton"], b.stats()["root_skeleton"]
    assert abs(ka - kb) <= 0.03 * kb
    la = [lv["max_k"] for lv in a.stats()["per_level"]]
    lb = [lv["max_k"] for lv in b.stats()["per_level"]]
    assert all(abs(x - y) <= 0.03 * y + 2 for x, y in zip(la, lb))


def test_mixed_fp32_factors_option(c1, monkeypatch):
    """SKEL_MIXED_FACTORS=fp32: elimination and factors in FP32 as well;
    still the same accuracy after GMRES on the 2048-node case."""
    wl, g, f, A, x = c1
    monkeypatch.setenv("SKEL_MIXED_FACTORS", "fp32")
    s = _mixed(wl)
    monkeypatch.delenv("SKEL_MIXED_FACTORS")
    s.factor()
    assert s.stats()["factor_storage"] == "fp32"
    assert_solution_close(s.solve(f), x, wl, TOL)
    assert s.stats()["gmres_iters"] <= 6


def test_mixed_update_equals_fresh_bitwise(c1):
    from gpu_util import to_device
    wl = c1[0]
    s = _mixed(wl)
    s.factor()
    moved = W.move_hole(wl, 1, (-0.01, 0.006))
    ids = np.arange(wl.node_slice(1).start, wl.node_slice(1).stop)
    s.update_moved_nodes(ids, to_device(moved))
    fresh = _mixed(moved)
    fresh.factor()
    rhs = np.random.default_rng(8).standard_normal(wl.n_unknowns)
    assert np.array_equal(s.solve(rhs), fresh.solve(rhs))


def test_solve_multi_rhs_and_adjoint(c1, c1_solver):
    wl, g, f, A, x = c1
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal((A.shape[0], 3))
    assert_solution_close(c1_solver.solve(rhs), np.linalg.solve(A, rhs), wl,
                          TOL)
    assert_solution_close(c1_solver.solve_adjoint(rhs),
                          np.linalg.solve(A.T, rhs), wl, TOL, "adjoint")


@pytest.mark.parametrize("n_outer,n_hole,nhole", [(2100, 901, 1),
                                                   (30000, 611, 16)])
def test_operator_apply_ragged_ranges(n_outer, n_hole, nhole):
    """The FP64 operator (symmetric pair sums over ranges of 128-point
    blocks) at node counts that leave a ragged last block and range, two
    right-hand sides: rows sampled across every range (the ragged tail
    included) match the oracle's rows to rounding, and two applies agree
    bit for bit.  The transposed operator satisfies the adjoint identity,
    and the double-float operator matches the FP64 one."""
    import torch
    if nhole == 1:
        wl = W.star1(n_outer=n_outer, n_hole=n_hole)
    else:
        wl = W.star16(n_outer=n_outer, n_hole=n_hole)
    assert wl.N % 128 != 0
    g = oracle.quadrature(wl)
    s = solver(wl)
    rng = np.random.default_rng(17)
    x = rng.standard_normal((wl.n_unknowns, 2))
    y = s.matvec(x)
    y2 = s.matvec(x)
    assert np.array_equal(np.asarray(y), np.asarray(y2))
    n2 = 2 * wl.N
    rows = np.unique(np.concatenate([
        rng.choice(n2, 96, replace=False), np.arange(n2 - 300, n2 + 3 * wl.p),
        np.arange(0, 8)]))
    yo = oracle.dense_matvec_rows(g, x, rows)
    assert rel(np.asarray(y)[rows], yo) < 1e-13
    # the transposed operator: <v, A x> = <A^T v, x> per column, and bit
    # for bit run to run
    v = rng.standard_normal((wl.n_unknowns, 2))
    at = np.asarray(s.matvec_adjoint(v))
    assert np.array_equal(at, np.asarray(s.matvec_adjoint(v)))
    for c in range(2):
        lhs = float(v[:, c] @ np.asarray(y)[:, c])
        rhs = float(at[:, c] @ x[:, c])
        scale = np.linalg.norm(v[:, c]) * np.linalg.norm(np.asarray(y)[:, c])
        assert abs(lhs - rhs) < 1e-13 * scale
    # the double-float operator (symmetric sums over ranges of curve-aligned
    # blocks) and its transpose against the FP64 ones, bit for bit run to run
    z = np.asarray(s.matvec_df(x))
    assert np.array_equal(z, np.asarray(s.matvec_df(x)))
    assert rel(z, np.asarray(y)) < 2e-13
    zt = np.asarray(s.matvec_adjoint_df(v))
    assert np.array_equal(zt, np.asarray(s.matvec_adjoint_df(v)))
    assert rel(zt, at) < 2e-13
    s.close()


def test_interior_velocity(c1, c1_solver):
    wl, g, f, A, x = c1
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    xs = c1_solver.solve(f)
    u = c1_solver.eval_velocity(xs, tx, ty)[:, :, 0]
    uo = oracle.interior_velocity(g, x, tx, ty)[:, :, 0]
    assert_velocity_close(u, uo, TOL)
    ue = oracle.point_force_velocity(tx, ty, wl.src_xy[0], wl.src_f[0])
    assert_velocity_close(u, ue, TOL)
    # evaluation alone matches to rounding on the same density
    u2 = c1_solver.eval_velocity(x, tx, ty)[:, :, 0]
    assert rel(u2, uo) < 1e-13


def test_agrees_with_oracle_skeletonization(c1):
    wl, g, f, A, x = c1
    fac = oracle.factor(wl)
    xo = oracle.solve(fac, f)
    s = solver(wl)
    s.factor()
    assert_solution_close(s.solve(f), xo, wl, TOL)
    st = s.stats()
    # same tree as the oracle (built independently from the same rules)
    assert st["levels"] == fac.tree.L
    assert st["boxes"] == len(fac.tree.boxes)


@pytest.mark.parametrize("case", ["no_holes", "single_leaf", "deep_tree",
                                  "three_holes"])
def test_edge_geometries(case):
    if case == "no_holes":
        wl = W.custom([W.star(1.0, 0.2, 5)], [700], n_targets=16,
                      leaf_size=32)
    elif case == "single_leaf":
        wl = W.custom([W.star(1.0, 0.2, 5), W.circle(0.2, (0.3, 0.1),
                                                      ccw=False)],
                      [40, 20], n_targets=0, leaf_size=64)
    elif case == "deep_tree":
        wl = W.custom([W.star(1.0, 0.2, 5), W.circle(0.2, (0.3, 0.1),
                                                      ccw=False),
                       W.ellipse(0.12, 0.07, 0.4, (-0.45, -0.2))],
                      [160, 48, 48], n_targets=0, leaf_size=8)
    else:
        wl = W.custom([W.star(1.0, 0.2, 5), W.circle(0.2, (0.3, 0.1),
                                                      ccw=False),
                       W.ellipse(0.15, 0.08, 0.7, (-0.4, -0.3)),
                       W.circle(0.1, (-0.3, 0.45), ccw=False)],
                      [1000, 300, 301, 157], n_targets=0, leaf_size=24)
    g = oracle.quadrature(wl)
    A = oracle.dense_system(g)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal((A.shape[0], 2))
    s = solver(wl)
    s.factor()
    assert_solution_close(s.solve(rhs), np.linalg.solve(A, rhs), wl, TOL)
    assert_solution_close(s.solve_adjoint(rhs), np.linalg.solve(A.T, rhs),
                          wl, TOL, "adjoint")


def test_update_equals_fresh_factorization_bitwise(c1):
    wl, g, f, A, x = c1
    s = solver(wl)
    s.factor()
    moved = W.move_hole(wl, 1, (0.012, -0.007))
    ids = np.arange(wl.node_slice(1).start, wl.node_slice(1).stop)
    from gpu_util import to_device
    s.update_moved_nodes(ids, to_device(moved))
    st = s.stats()
    assert 0 < st["last_dirty"] < st["last_boxes"]
    fresh = solver(moved)
    fresh.factor()
    g2 = oracle.quadrature(moved)
    f2 = oracle.boundary_data(g2, wl.src_xy, wl.src_f)
    a, b = s.solve(f2), fresh.solve(f2)
    assert np.array_equal(a, b)
    x2 = np.linalg.solve(oracle.dense_system(g2), f2)
    assert_solution_close(a, x2, wl, TOL)


def test_repeated_updates_on_many_holes():
    """Several successive hole moves on the 16-hole geometry at a quarter of
    its node counts: after every update the solve and the adjoint solve equal
    those of a fresh factorization bit for bit (Sec. 2.8), and the dense
    oracle residual stays at the solver tolerance."""
    from gpu_util import to_device
    wl = W.scaled(W.star16(), 4, n_targets=16)
    s = solver(wl)
    s.factor()
    cur = wl
    rng = np.random.default_rng(9)
    for h, d in W.random_moves(wl, 3, seed=5):
        cur = W.move_hole(cur, h, d)
        sl = cur.node_slice(h)
        s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(cur))
        fresh = solver(cur)
        fresh.factor()
        rhs = rng.standard_normal((cur.n_unknowns, 2))
        assert np.array_equal(s.solve(rhs), fresh.solve(rhs))
        assert np.array_equal(s.solve_adjoint(rhs), fresh.solve_adjoint(rhs))
        fresh.close()
    g = oracle.quadrature(cur)
    f = oracle.boundary_data(g, cur.src_xy, cur.src_f)
    x = s.solve(f)
    rows = np.random.default_rng(1).choice(cur.n_unknowns, 16, replace=False)
    res = oracle.dense_matvec_rows(g, x, rows)[:, 0] - f[rows, 0]
    assert np.abs(res).max() < TOL * np.abs(f).max()


def _scaled_hole(w, h, f):
    """Hole h (1-based) scaled by f about its centre: the nodes and their
    derivatives change, the centre does not."""
    from dataclasses import replace
    sl = w.node_slice(h)
    cx, cy = w.centers[h - 1]
    out = {}
    for k, c in (("x", cx), ("y", cy)):
        a = np.array(getattr(w, k))
        a[sl] = c + f * (a[sl] - c)
        out[k] = a
    for k in ("dx", "dy", "ddx", "ddy"):
        a = np.array(getattr(w, k))
        a[sl] *= f
        out[k] = a
    return replace(w, **out)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bordered_sweep_after_partial_changes(prec):
    """Updates that change the bordered columns in part (Sec. 3.2): a hole
    whose centre alone moves (its Stokeslet / rotlet columns change at every
    node, no box is recompressed), a hole scaled about a fixed centre (boxes
    recompressed, the centre columns kept), then a rigid move.  Each must
    equal a fresh factorization bit for bit, solve and adjoint solve."""
    from dataclasses import replace

    from gpu_util import to_device
    wl = W.scaled(W.star16(), 4, n_targets=16)
    mk = _mixed if prec == "mixed" else solver
    s = mk(wl)
    s.factor()
    rng = np.random.default_rng(21)
    c = wl.centers.copy()
    c[2] += (1e-3, -5e-4)
    cur = replace(wl, centers=c)
    steps = [("centre", cur, 3)]
    cur = _scaled_hole(cur, 5, 0.97)
    steps.append(("scale", cur, 5))
    cur = W.move_hole(cur, 3, (0.004, 0.002))
    steps.append(("move", cur, 3))
    for name, cur, h in steps:
        sl = cur.node_slice(h)
        ids = np.arange(sl.start, sl.stop) if name != "centre" else \
            np.arange(0, 0)
        s.update_moved_nodes(ids, to_device(cur))
        if name == "centre":
            assert s.stats()["last_dirty"] == 0
        fresh = mk(cur)
        fresh.factor()
        rhs = rng.standard_normal((cur.n_unknowns, 2))
        assert np.array_equal(s.solve(rhs), fresh.solve(rhs)), name
        assert np.array_equal(s.solve_adjoint(rhs),
                              fresh.solve_adjoint(rhs)), name
        fresh.close()
    s.close()


def test_solve_before_factor_is_an_error(c1):
    import paper_2001_11619_gb300 as skel
    s = solver(c1[0])
    with pytest.raises(skel.SkelError) as e:
        s.solve(c1[2])
    assert e.value.code == -8


@pytest.mark.slow
def test_star16_full_size_sampled():
    """The 32768-node, 16-hole workload at full size: residual rows of the
    bordered system computed one by one by the oracle, and the interior
    velocity against the exact point-force field."""
    wl = W.star16()
    s = solver(wl)
    s.factor()
    f = s.point_force_rhs(wl.src_xy, wl.src_f)
    xs = s.solve(f)
    g = oracle.quadrature(wl)
    fo = oracle.boundary_data(g, wl.src_xy, wl.src_f)
    assert rel(f, fo) < 1e-13
    rows = np.random.default_rng(4).choice(wl.n_unknowns, 24, replace=False)
    res = oracle.dense_matvec_rows(g, xs, rows)[:, 0] - fo[rows, 0]
    assert np.abs(res).max() < TOL * np.abs(fo).max()
    tx, ty = wl.targets[:256, 0], wl.targets[:256, 1]
    u = s.eval_velocity(xs, tx, ty)[:, :, 0]
    ue = oracle.point_force_velocity(tx, ty, wl.src_xy[0], wl.src_f[0])
    assert_velocity_close(u, ue, TOL)
    uo = oracle.interior_velocity(g, xs, tx[:32], ty[:32])[:, :, 0]
    assert rel(u[:32], uo) < 1e-13


@pytest.mark.slow
def test_star16_full_size_mixed():
    """The mixed form on the full 16-hole workload: residual rows from the
    oracle and the interior velocity against the exact field."""
    wl = W.star16()
    s = _mixed(wl, gmres_tol=1e-12)
    s.factor()
    f = s.point_force_rhs(wl.src_xy, wl.src_f)
    xs = s.solve(f)
    assert s.stats()["gmres_iters"] <= 6
    rng = np.random.default_rng(13)
    v = rng.standard_normal(wl.n_unknowns)
    assert rel(s.matvec_df(v), s.matvec(v)) < 2e-13
    g = oracle.quadrature(wl)
    fo = oracle.boundary_data(g, wl.src_xy, wl.src_f)
    rows = np.random.default_rng(4).choice(wl.n_unknowns, 24, replace=False)
    res = oracle.dense_matvec_rows(g, xs, rows)[:, 0] - fo[rows, 0]
    assert np.abs(res).max() < TOL * np.abs(fo).max()
    tx, ty = wl.targets[:256, 0], wl.targets[:256, 1]
    u = s.eval_velocity(xs, tx, ty)[:, :, 0]
    ue = oracle.point_force_velocity(tx, ty, wl.src_xy[0], wl.src_f[0])
    assert_velocity_close(u, ue, TOL)


def _sampled_checks(wl, s, xs, nrows=12, nt=64):
    """Residual rows of the bordered system computed one by one by the
    oracle, and interior velocities against the exact point-force field,
    for every right-hand side."""
    g = oracle.quadrature(wl)
    nrhs = xs.shape[1]
    fo = oracle.boundary_data(g, wl.src_xy[:nrhs], wl.src_f[:nrhs])
    rows = np.random.default_rng(4).choice(wl.n_unknowns, nrows,
                                           replace=False)
    res = oracle.dense_matvec_rows(g, xs, rows) - fo[rows]
    assert np.abs(res).max() < TOL * np.abs(fo).max()
    tx, ty = wl.targets[:nt, 0].copy(), wl.targets[:nt, 1].copy()
    u = s.eval_velocity(xs, tx, ty)
    for c in range(nrhs):
        ue = oracle.point_force_velocity(tx, ty, wl.src_xy[c], wl.src_f[c])
        assert_velocity_close(u[:, :, c], ue, TOL)


@pytest.mark.slow
def test_quad64_full_size():
    """The 131072-node quadrant geometry with 64 clustered holes (leaf 128):
    the top-level boxes hold whole holes, so X_RR conditioning moves
    indices into the skeleton (Sec. 2.2 remark); 8 right-hand sides in the
    FP64 form, one in the mixed form, and a moved hole whose update equals
    a fresh factorization bit for bit."""
    from gpu_util import to_device
    wl = W.quad64()
    s = solver(wl)
    s.factor()
    assert sum(lv["moved"] for lv in s.stats()["per_level"]) > 0
    f = s.point_force_rhs(wl.src_xy, wl.src_f)
    xs = s.solve(f)
    _sampled_checks(wl, s, xs)
    m = _mixed(wl, id_tol=3e-7, gmres_tol=1e-12)
    m.factor()
    xm = m.solve(f[:, :1])
    assert m.stats()["gmres_iters"] <= 6
    _sampled_checks(wl, m, xm)
    m.close()
    h, d = W.random_moves(wl, 1, seed=3)[0]
    moved = W.move_hole(wl, h, d)
    sl = moved.node_slice(h)
    s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(moved))
    fresh = solver(moved)
    fresh.factor()
    assert np.array_equal(s.solve(f), fresh.solve(f))


@pytest.mark.slow
def test_star256_full_size_fp64():
    """The 1048576-node, 256-hole star geometry in the FP64 form with the
    32-column batched solve; sampled residual rows and velocities."""
    wl = W.star256()
    s = solver(wl)
    s.factor()
    f = s.point_force_rhs(wl.src_xy, wl.src_f)
    xs = s.solve(f)
    assert xs.shape[1] == 32
    _sampled_checks(wl, s, xs, nrows=8, nt=32)


def test_tuning_parameters_and_autotuner(c1):
    """Launch-shape parameters: defaults, validation, re-factor required
    after a change, the same solution (to rounding) under every setting,
    and the autotuner leaving a factored solver."""
    import paper_2001_11619_gb300 as skel
    from paper_2001_11619_gb300 import autotune
    wl, g, f, A, x = c1
    s = solver(wl)
    t0 = s.get_tuning()
    assert {k: t0[k] for k in ("cluster_min_n", "cluster_level_boxes",
                               "sweep_rhs_chunk")} == {
        "cluster_min_n": 160, "cluster_level_boxes": 76,
        "sweep_rhs_chunk": 16}
    with pytest.raises(skel.SkelError):
        s.set_tuning(sweep_rhs_chunk=5)
    with pytest.raises(skel.SkelError):
        s.set_tuning(no_such_key=1)
    s.factor()
    ref = s.solve(f)
    s.set_tuning(cluster_min_n=64, cluster_level_boxes=0)
    with pytest.raises(skel.SkelError):
        s.solve(f)  # factors dropped until the next factor()
    s.factor()
    assert rel(s.solve(f), ref) < 1e-11
    # mid-size boxes on 4-CTA clusters
    s.set_tuning(cluster_min_n=160, cluster_mid_min_n=48,
                 cluster_mid_level_boxes=1000)
    s.factor()
    assert s.stats()["per_level"][-1]["cluster_boxes"] > 0
    assert rel(s.solve(f), ref) < 1e-11
    import torch
    fd = torch.tensor(f, device="cuda")
    res = autotune.tune(s, fd, candidates={"cluster_min_n": (64, 160),
                                           "sweep_rhs_chunk": (4, 16)},
                        repeats=1)
    assert set(res["config"]) == set(s.TUNING_KEYS)
    assert res["ms"] > 0 and len(res["trials"]) == 3
    assert s.get_tuning() == res["config"]
    assert_solution_close(s.solve(f), x, wl, TOL)
    s.close()


def test_mixed_double_float_convergence_test(c1):
    """At gmres_tol >= 1e-11 the double-float operator's residual decides
    convergence, read from the GMRES recurrence once a cycle meets its
    inner target (no FP64 operator apply in the solve); the FP64 residual
    is still below the tolerance and the solution meets the 1e-10 target
    entry by entry.  gmres_fp64_check restores the FP64 test,
    which needs at least one FP64 apply."""
    wl, g, f, A, x = c1
    s = _mixed(wl, gmres_tol=1e-11)
    s.factor()
    s.set_timing(True)
    xs = s.solve(f)
    st = s.stats()
    assert st["gmres_check"] == "df"
    assert st["gmres_recurrence"] == 1
    assert "matvec" not in st["kernels"]
    assert st["kernels"]["matvec_df"]["launches"] > 0
    assert_solution_close(xs, x, wl, TOL)
    r = np.asarray(s.matvec(xs)) - f
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-11 * 1.05
    s.set_gmres_fp64_check(True)
    s.set_timing(True)
    x2 = s.solve(f)
    st = s.stats()
    assert st["gmres_check"] == "fp64"
    assert st["gmres_recurrence"] == 0
    assert st["kernels"]["matvec"]["launches"] >= 1
    assert_solution_close(x2, x, wl, TOL)
    s.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quad64_ten_consecutive_moves(prec):
    """The 131072-node, 64 clustered-hole workload (Table 1's setting of
    repeated hole moves): ten moved holes in a row, each update equal to a
    fresh factorization of the moved geometry bit for bit (Sec. 2.8), then
    oracle residual rows and the exact field on the last geometry."""
    from gpu_util import to_device
    wl = W.quad64()
    mk = (lambda w: _mixed(w, id_tol=3e-7, gmres_tol=1e-11)) \
        if prec == "mixed" else solver
    s = mk(wl)
    s.factor()
    cur = wl
    rhs = np.random.default_rng(23).standard_normal(wl.n_unknowns)
    for h, d in W.random_moves(wl, 10, seed=31):
        cur = W.move_hole(cur, h, d)
        sl = cur.node_slice(h)
        s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(cur))
        fresh = mk(cur)
        fresh.factor()
        assert np.array_equal(s.solve(rhs), fresh.solve(rhs))
        fresh.close()
    g = oracle.quadrature(cur)
    f = oracle.boundary_data(g, cur.src_xy[:2], cur.src_f[:2])
    xs = s.solve(f)
    _sampled_checks(cur, s, np.asarray(xs))
    s.close()


@pytest.mark.slow
def test_star256_full_size_mixed_and_update():
    """The 1M-node, 256-hole workload in the mixed form: factor, a solve
    checked against oracle residual rows and the exact field, then a moved
    hole whose update equals a fresh factorization bit for bit.  (One
    column: each mixed solve here is GMRES with O(N^2) double-float
    products, about 20 s per column.)"""
    from gpu_util import to_device
    wl = W.star256()
    s = _mixed(wl, gmres_tol=1e-11)
    s.factor()
    f = s.point_force_rhs(wl.src_xy[:1], wl.src_f[:1])
    xs = s.solve(f)
    assert s.stats()["gmres_iters"] <= 6
    _sampled_checks(wl, s, np.asarray(xs).reshape(-1, 1), nrows=6, nt=32)
    h, d = W.random_moves(wl, 1, seed=5)[0]
    moved = W.move_hole(wl, h, d)
    sl = moved.node_slice(h)
    s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(moved))
    assert 0 < s.stats()["last_dirty"] < s.stats()["last_boxes"]
    fresh = _mixed(moved, gmres_tol=1e-11)
    fresh.factor()
    f2 = fresh.point_force_rhs(wl.src_xy[:1], wl.src_f[:1])
    assert np.array_equal(s.solve(f2), fresh.solve(f2))
    fresh.close()
    s.close()


def test_top_block_blocked_solve_matches_columnwise():
    """With several right-hand sides and a top block of at least 1024
    unknowns the top-block solve runs as blocked triangular solves over all
    SMs (one CTA per column below that), and the border products run 32
    right-hand sides per CTA.  On the 32768-node case (top block 1229, 48
    border columns: a full and a ragged tile) a 37-column solve and adjoint
    solve (two right-hand-side tiles, the second ragged) agree with the
    same columns solved one at a time, and their residual rows with the
    oracle's."""
    wl = W.star16()
    s = solver(wl)
    s.factor()
    assert s.stats()["root_skeleton"] + 3 * wl.p >= 1024
    rng = np.random.default_rng(41)
    nr = 37
    rhs = rng.standard_normal((wl.n_unknowns, nr))
    for fn in (s.solve, s.solve_adjoint):
        xb = np.asarray(fn(rhs))
        xc = np.stack([np.asarray(fn(rhs[:, c])) for c in range(nr)], axis=1)
        assert rel(xb, xc) < 1e-12
    g = oracle.quadrature(wl)
    xb = np.asarray(s.solve(rhs[:, :2]))
    rows = rng.choice(wl.n_unknowns, 8, replace=False)
    res = oracle.dense_matvec_rows(g, xb, rows) - rhs[rows, :2]
    assert np.abs(res).max() < TOL * np.abs(rhs).max() * 10
    s.close()
