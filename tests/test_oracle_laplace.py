"""Pins for the Laplace Neumann oracle (oracle.laplace), CPU only: the
constant-density identity on a circle, the diagonal limit along a curve,
the one-dimensional null space that N completes, recovery of closed-form
harmonic fields from their flux, and the paper's flux data (0 on the outer
curve, +1 and -1 on two holes)."""
import numpy as np

import workloads as W
from oracle import laplace as L


def _geom(curves, counts):
    w = W.custom(curves, counts, n_targets=24, seed=3)
    return w, L.quadrature(w)


def test_constant_density_on_the_unit_circle():
    w, g = _geom([W.circle(1.0)], [256])
    d = L.d_entries(g, np.arange(g.N), np.arange(g.N))
    # (x - y).n(x) = |x - y|^2 / 2 on the unit circle: D 1 = -1/2 exactly
    assert np.abs(d.sum(1) + 0.5).max() < 1e-13


def test_diagonal_limit_along_a_curve():
    w, g = _geom([W.ellipse(1.0, 0.5, 0.3, (0.0, 0.0), ccw=True)], [8192])
    i = np.arange(0, g.N, 97)
    diag = L.d_entries(g, i, i).diagonal() / g.w[i]
    nxt = np.array([L.d_entries(g, [k], [(k + 1) % g.N])[0, 0]
                    / g.w[(k + 1) % g.N] for k in i])
    # the kernel at the neighbouring node tends to the diagonal value
    assert np.abs(nxt - diag).max() < 2e-3 * np.abs(diag).max()


def _holes():
    return [W.star(1.0, 0.2, 5),
            W.ellipse(0.15, 0.1, 0.4, (0.35, 0.1)),
            W.ellipse(0.12, 0.08, -0.3, (-0.35, -0.15))]


def test_one_dimensional_null_space_completed_by_n():
    w, g = _geom(_holes(), [400, 160, 160])
    idx = np.arange(g.N)
    a0 = L.d_entries(g, idx, idx) + 0.5 * np.eye(g.N)
    sv = np.linalg.svd(a0, compute_uv=False)
    assert sv[-1] < 1e-12 * sv[0]
    assert sv[-2] > 1e-3 * sv[0]
    sa = np.linalg.svd(L.dense_system(g), compute_uv=False)
    assert sa[-1] > 1e-3 * sa[0]


def test_flux_recovers_harmonic_fields():
    """u = 0.7 x - 0.3 y + log sources outside Gamma_0 and inside the holes:
    solving with its flux gives S mu = u up to a constant in Omega."""
    w, g = _geom(_holes(), [1536, 512, 512])
    src = np.array([[2.1, 0.4], [-1.7, -1.6], [0.35, 0.1], [-0.35, -0.15]])
    q = np.array([0.8, -1.1, 0.6, -0.4])
    f = 0.7 * g.nx - 0.3 * g.ny + L.source_flux(g, src, q)
    mu = L.dense_solve(g, f)
    assert abs(np.dot(g.w, mu)) < 1e-12 * np.abs(mu).max()
    tx, ty = w.targets[:, 0], w.targets[:, 1]
    u = L.single_layer(g, mu, tx, ty)
    ue = 0.7 * tx - 0.3 * ty + L.source_potential(tx, ty, src, q)
    du, due = u - u[0], ue - ue[0]
    assert np.abs(du - due).max() < 1e-10 * np.abs(due).max()


def test_paper_flux_data_is_solvable():
    """The paper's data: 0 on Gamma_0, +1 on hole 1, -1 on hole 2 (two
    congruent holes): total flux 0, int mu = 0, and mu solves the
    uncompleted equation."""
    curves = [W.star(1.0, 0.2, 5), W.ellipse(0.15, 0.1, 0.0, (0.35, 0.1)),
              W.ellipse(0.15, 0.1, 0.0, (-0.35, -0.15))]
    w, g = _geom(curves, [800, 200, 200])
    f = np.where(g.comp == 1, 1.0, np.where(g.comp == 2, -1.0, 0.0))
    assert abs(np.dot(g.w, f)) < 1e-12
    mu = L.dense_solve(g, f)
    assert abs(np.dot(g.w, mu)) < 1e-12 * np.abs(mu).max()
    idx = np.arange(g.N)
    r = (L.d_entries(g, idx, idx) + 0.5 * np.eye(g.N)) @ mu - f
    assert np.abs(r).max() < 1e-11
