"""Pins for the oracle's exact discrete system (O-1) against closed forms,
invariants and the paper's own analytic test.  CPU only."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import stokes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dofs(n):
    return np.arange(2 * n)


def test_unit_circle_constant_density():
    """Jump relation (Eq. jump): inside the unit circle the double layer of a
    constant density c is -c, so the discrete boundary operator maps c to
    -c/2 (trapezoid rule exact here, diagonal limit included)."""
    w = W.custom([W.circle(1.0)], [96], n_targets=0)
    g = oracle.quadrature(w)
    K = oracle.k_entries(g, _dofs(96), _dofs(96))
    c = np.tile([0.3, -0.7], 96)
    assert np.abs(K @ c + 0.5 * c).max() < 1e-14


def test_double_layer_of_constant_at_centre():
    """D[c](centre) = -c: with r = -y, r.n = -R, and the mean of y y^T over
    the circle R^2 I / 2 (Eq. stokesbie)."""
    R, ctr = 0.7, np.array([0.2, -0.1])
    w = W.custom([W.circle(R, tuple(ctr))], [64], n_targets=0)
    g = oracle.quadrature(w)
    c = np.array([1.3, -0.4])
    sol = np.tile(c, 64)
    u = oracle.interior_velocity(g, sol, [ctr[0]], [ctr[1]])[0, :, 0]
    assert np.abs(u + c).max() < 1e-14


def test_diagonal_limit_along_curve():
    """The diagonal entry is the limit of D(x_i, gamma(t_i + d)) w as d -> 0
    on a curve of varying curvature (symmetric difference removes O(d))."""
    cv = W.ellipse(0.4, 0.15, 0.3, (0.1, 0.2), ccw=False)
    n = 64
    w = W.custom([W.circle(1.0), cv], [64, n], n_targets=0)
    g = oracle.quadrature(w)
    K = oracle.k_entries(g, np.arange(128, 128 + 2 * n),
                         np.arange(128, 128 + 2 * n))
    dt = 2 * np.pi / n
    for i in (0, 5, 17, 40):
        ti = -i * dt                     # the hole runs clockwise: p(-t)
        acc = np.zeros((2, 2))
        for d in (1e-3, -1e-3):
            x, y, dx, dy, *_ = cv.eval(np.array([ti + d]))
            sp = np.hypot(dx, dy)
            # orientation of the clockwise hole: gamma' = -p'
            snx, sny = -dy / sp, dx / sp
            blk = S.dl_blocks(np.array([g.x[64 + i]]), np.array([g.y[64 + i]]),
                              x, y, snx, sny, np.array([g.w[64 + i]]))
            acc += 0.5 * blk[0, 0]
        diag = K[2 * i:2 * i + 2, 2 * i:2 * i + 2]
        assert np.abs(diag - acc).max() < 1e-5 * np.abs(diag).max()


def _two_hole_geom():
    curves = [W.star(1.0, 0.2, 5), W.circle(0.2, (0.3, 0.1), ccw=False),
              W.ellipse(0.15, 0.08, 0.7, (-0.4, -0.3))]
    w = W.custom(curves, [300, 120, 120], n_targets=0)
    return w, oracle.quadrature(w)


def test_rigid_motions_span_the_null_space():
    """Eq. (null-space): (-1/2 I + D + N) Psi = 0 for the per-hole rigid
    motions, and there is no other null vector (the completion N removes the
    flux null vector, Eq. null-spaceop): exactly 3p singular values vanish."""
    w, g = _two_hole_geom()
    d = _dofs(g.N)
    A11 = oracle.a11_entries(g, d, d)
    Psi = oracle.psi_columns(g, d)
    assert np.abs(A11 @ (Psi / g.w.repeat(2)[:, None])).max() < 1e-13
    sv = np.linalg.svd(A11, compute_uv=False)
    assert np.sum(sv < 1e-12 * sv[0]) == 3 * g.p
    assert sv[-3 * g.p - 1] > 1e-3 * sv[0]
    A = oracle.dense_system(g)
    sv = np.linalg.svd(A, compute_uv=False)
    assert sv[-1] > 1e-5 * sv[0]          # bordered system: nonsingular


def test_psi_integrals_closed_form():
    """Psi^T mu are the integrals over hole i of mu_x, mu_y and x^perp.mu;
    for mu = x^perp on a circle of radius a about c they equal
    -2 pi a c_y, 2 pi a c_x and 2 pi a (a^2 + |c|^2)."""
    a, c = 0.2, np.array([0.3, 0.1])
    w = W.custom([W.circle(1.0), W.circle(a, tuple(c), ccw=False)],
                 [64, 80], n_targets=0)
    g = oracle.quadrature(w)
    d = _dofs(g.N)
    mu = np.stack([-g.y, g.x], axis=1).reshape(-1)
    mu[:128] = 0.0
    got = oracle.psi_columns(g, d).T @ mu
    want = [-2 * np.pi * a * c[1], 2 * np.pi * a * c[0],
            2 * np.pi * a * (a * a + c @ c)]
    assert np.allclose(got, want, rtol=1e-13, atol=1e-15)


def _traction_on_circle(vel, pres, c, rho=0.3, n=64, h=1e-5):
    """Force and torque exerted across a circle about c by the fluid outside
    it: int sigma n ds and int (x-c)^perp . sigma n ds, sigma = -p I +
    grad u + grad u^T (unit viscosity); grad u by central differences."""
    th = 2 * np.pi * np.arange(n) / n
    F = np.zeros(2)
    Tq = 0.0
    for t in th:
        nrm = np.array([np.cos(t), np.sin(t)])
        x = c + rho * nrm
        J = np.zeros((2, 2))
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            J[:, k] = (vel(x + e) - vel(x - e)) / (2 * h)
        sig = -pres(x) * np.eye(2) + J + J.T
        tr = sig @ nrm * (2 * np.pi * rho / n)
        F += tr
        r = x - c
        Tq += -r[1] * tr[0] + r[0] * tr[1]
    return F, Tq


def test_stokeslet_and_rotlet_strengths():
    """Sec. 3.1: a Stokeslet of strength alpha exerts total force alpha and
    no torque, a rotlet of strength beta total torque beta and no force; the
    fluid outside a circle about c therefore pulls on it with -alpha / -beta.
    (Pressure of the 2-D Stokeslet: alpha.r / (2 pi |r|^2); rotlet: 0.)"""
    c = np.array([0.1, -0.2])
    g = S.Geom(np.zeros(1), np.zeros(1), np.ones(1), np.zeros(1), np.ones(1),
               np.zeros(1), np.zeros(1, int), c[None, :])
    for a, strength in ((0, 1.7), (1, -0.6)):
        col = lambda x: oracle.h_columns(
            S.Geom(np.array([x[0]]), np.array([x[1]]), g.nx, g.ny, g.w,
                   g.kap, g.comp, g.centers), [0, 1])[:, a] * strength
        fvec = np.zeros(2)
        fvec[a] = strength
        pres = lambda x: fvec @ (x - c) / (2 * np.pi * ((x - c) @ (x - c)))
        F, Tq = _traction_on_circle(col, pres, c)
        assert np.allclose(F, -fvec, atol=1e-7)
        assert abs(Tq) < 1e-7
    beta = 0.9
    rot = lambda x: oracle.h_columns(
        S.Geom(np.array([x[0]]), np.array([x[1]]), g.nx, g.ny, g.w, g.kap,
               g.comp, g.centers), [0, 1])[:, 2] * beta
    F, Tq = _traction_on_circle(rot, lambda x: 0.0, c)
    assert np.abs(F).max() < 1e-7
    assert abs(Tq + beta) < 1e-7


def test_stokeslet_recovery_dense(star1, star1_dense):
    """Velocity from point forces outside Gamma_0 is recovered at interior
    targets (Eq. completed) to 1e-10; the flux constraint holds and the
    second block row gives lambda = Psi^T mu (Eq. backwardeq)."""
    g, f, sol = star1_dense
    tx, ty = star1.targets[:, 0], star1.targets[:, 1]
    u = oracle.interior_velocity(g, sol, tx, ty)[:, :, 0]
    ue = oracle.point_force_velocity(tx, ty, star1.src_xy[0], star1.src_f[0])
    assert np.abs(u - ue).max() < 1e-10 * np.abs(ue).max()
    mu = sol[:2 * g.N, 0].reshape(-1, 2)
    assert abs(np.sum(g.w * (g.nx * mu[:, 0] + g.ny * mu[:, 1]))) < 1e-12
    lam = oracle.psi_columns(g, _dofs(g.N)).T @ sol[:2 * g.N, 0]
    assert np.allclose(lam, sol[2 * g.N:, 0], atol=1e-13)


def test_stokeslet_recovery_with_forces_inside_holes():
    """Point forces inside the holes need the Stokeslet columns of H: the
    double layer alone cannot represent them (Sec. 3.1)."""
    curves = [W.star(1.0, 0.2, 5), W.circle(0.2, (0.3, 0.1), ccw=False),
              W.ellipse(0.15, 0.08, 0.7, (-0.4, -0.3))]
    w = W.custom(curves, [1024, 384, 384], n_targets=64, seed=3)
    g = oracle.quadrature(w)
    sxy = np.array([[[2.0, 0.5], [0.31, 0.12], [-0.41, -0.29]]])
    sf = np.array([[[1.0, -0.5], [0.3, 0.8], [-0.7, 0.4]]])
    f = oracle.boundary_data(g, sxy, sf)
    sol = oracle.dense_solve(g, f)
    tx, ty = w.targets[:, 0], w.targets[:, 1]
    u = oracle.interior_velocity(g, sol, tx, ty)[:, :, 0]
    ue = oracle.point_force_velocity(tx, ty, sxy[0], sf[0])
    assert np.abs(u - ue).max() < 1e-10 * np.abs(ue).max()
    # the forces inside the holes reappear as the Stokeslet strengths alpha
    lam = sol[2 * g.N:, 0].reshape(2, 3)
    assert np.allclose(lam[:, :2], sf[0, 1:], atol=1e-9)


def _couette():
    R1, R2, V1, V2, A, B = np.loadtxt(os.path.join(GOLDEN, "couette.txt"))
    assert abs(A * R1 + B / R1 - V1) < 1e-15
    assert abs(A * R2 + B / R2 - V2) < 1e-15
    curves = [W.circle(R2), W.circle(R1, ccw=False)]
    w = W.custom(curves, [512, 256], n_targets=0)
    g = oracle.quadrature(w)
    f = np.zeros((2 * g.N + 3, 1))
    V = np.where(g.comp == 0, V2, V1)
    r = np.hypot(g.x, g.y)
    f[:2 * g.N:2, 0] = -V * g.y / r
    f[1:2 * g.N:2, 0] = V * g.x / r
    rr, tt = np.meshgrid(np.linspace(R1 + 0.1, R2 - 0.1, 9),
                         np.linspace(0, 2 * np.pi, 13, endpoint=False))
    tx, ty = (rr * np.cos(tt)).ravel(), (rr * np.sin(tt)).ravel()
    ut = A * rr.ravel() + B / rr.ravel()
    ue = np.stack([-ut * np.sin(tt.ravel()), ut * np.cos(tt.ravel())], 1)
    return w, g, f, tx, ty, ue


def test_couette_dense():
    """The paper's analytic test (Sec. 4.1): concentric circles with
    tangential boundary velocities; the rotlet carries the torque."""
    w, g, f, tx, ty, ue = _couette()
    sol = oracle.dense_solve(g, f)
    u = oracle.interior_velocity(g, sol, tx, ty)[:, :, 0]
    assert np.abs(u - ue).max() < 1e-10 * np.abs(ue).max()


def test_dense_matvec_rows_consistent(star1_dense):
    g, f, sol = star1_dense
    rows = [0, 1, 777, 2 * g.N - 1, 2 * g.N, 2 * g.N + 2]
    r = oracle.dense_matvec_rows(g, sol, rows)[:, 0] - f[rows, 0]
    assert np.abs(r).max() < 1e-12
