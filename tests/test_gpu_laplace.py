"""The Laplace Neumann variant (Sec. 4.4.1: steady heat flow with flux
data, single-layer representation, no bordering) through the same engine,
against the oracle's dense solve and closed forms:
- the operator apply against the dense matrix;
- the solve, adjoint solve and potential against the dense LU at 2048
  nodes, to the 1e-10 bar;
- recovery of a closed-form harmonic field from its flux at 16384 nodes
  (the paper's size);
- a hole move equal to a fresh factorization bit for bit;
- the Stokes-only calls refused."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel, to_device

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _solver(wl, **kw):
    import paper_2001_11619_gb300 as skel
    kw.setdefault("leaf_size", wl.leaf_size)
    kw.setdefault("id_tol", 1e-12)
    return skel.Solver(to_device(wl), kernel=skel.LAPLACE, **kw)


@pytest.fixture(scope="module")
def small():
    from oracle import laplace as L
    wl = W.heat2(N=2048, n_targets=64)
    g = L.quadrature(wl)
    A = L.dense_system(g)
    return wl, g, A


def test_operator_apply_matches_dense(small):
    wl, g, A = small
    s = _solver(wl)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((g.N, 2))
    assert s.n == g.N
    assert rel(s.matvec(x), A @ x) < 1e-13
    s.close()


def test_solve_and_potential_match_dense(small):
    from oracle import laplace as L
    wl, g, A = small
    s = _solver(wl)
    s.factor()
    st = s.stats()
    assert st["root_skeleton"] < g.N
    f = W.heat_flux(wl)
    mu = s.solve(f)
    mu_o = L.dense_solve(g, f)
    assert rel(mu, mu_o) < TOL
    rng = np.random.default_rng(2)
    b = rng.standard_normal((g.N, 3))
    assert rel(s.solve(b), np.linalg.solve(A, b)) < TOL
    assert rel(s.solve_adjoint(b), np.linalg.solve(A.T, b)) < TOL
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    u = s.eval_potential(mu, tx, ty)[:, 0]
    assert rel(u, L.single_layer(g, mu_o, tx, ty)) < TOL
    # the paper's data has zero total flux: int mu = 0
    assert abs(np.dot(g.w, mu)) < 1e-11 * np.abs(mu).max()
    s.close()


def test_harmonic_field_from_its_flux_at_full_size():
    """u = 0.7 x - 0.3 y + log sources outside Gamma_0 and inside both
    holes, at 16384 nodes: S mu = u up to a constant at interior targets,
    and the GPU operator residual is at the solver tolerance."""
    import torch
    from oracle import laplace as L
    wl = W.heat2(N=16384, n_targets=256)
    g = L.quadrature(wl)
    src = np.array([[2.1, 0.4], [-1.7, -1.6], list(wl.centers[0]),
                    list(wl.centers[1])])
    q = np.array([0.8, -1.1, 0.6, -0.4])
    f = 0.7 * g.nx - 0.3 * g.ny + L.source_flux(g, src, q)
    s = _solver(wl)
    s.factor()
    fd = torch.tensor(f, device="cuda")
    mu = s.solve(fd)
    r = s.matvec(mu) - fd
    assert float(torch.linalg.norm(r) / torch.linalg.norm(fd)) < 1e-11
    tx, ty = wl.targets[:, 0], wl.targets[:, 1]
    u = s.eval_potential(mu, tx, ty)[:, 0].cpu().numpy()
    ue = 0.7 * tx - 0.3 * ty + L.source_potential(tx, ty, src, q)
    du, due = u - u[0], ue - ue[0]
    assert np.abs(du - due).max() < 1e-9 * np.abs(due).max()
    s.close()


def test_hole_move_equals_fresh_factorization():
    import torch
    wl = W.heat2(N=4096, n_targets=16)
    s = _solver(wl)
    s.factor()
    moved = W.move_hole(wl, 2, (0.01, -0.006))
    sl = moved.node_slice(2)
    s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(moved))
    st = s.stats()
    assert 0 < st["last_dirty"] < st["last_boxes"]
    fresh = _solver(moved)
    fresh.factor()
    f = torch.tensor(W.heat_flux(moved), device="cuda")
    assert torch.equal(s.solve(f), fresh.solve(f))
    s.close()
    fresh.close()


def test_stokes_only_calls_are_refused(small):
    import paper_2001_11619_gb300 as skel
    wl, g, A = small
    with pytest.raises(skel.SkelError):
        skel.Solver(to_device(wl), kernel=skel.LAPLACE, precision=skel.MIXED)
    s = _solver(wl)
    s.factor()
    with pytest.raises(skel.SkelError):
        s.point_force_rhs(wl.src_xy, wl.src_f)
    with pytest.raises(skel.SkelError):
        s.matvec_adjoint(np.zeros(g.N))
    s.close()
