"""O-1 for the Laplace Neumann variant of the paper's Sec. 4.4.1 experiment
(steady heat flow with flux data): the exact discrete single-layer system,
FP64, dense.  Test infrastructure only (see the package docstring).

The paper represents u = S mu with the single layer
    S mu(x) = -(1/2 pi) int_Gamma log|x - y| mu(y) dy
and solves its boundary equation with the kernel
    D mu(x) = -(1/2 pi) int_Gamma (x - y).n(x) / |x - y|^2 mu(y) dy,
i.e. the normal derivative of S at the target.  The integral operator is
full rank after the completion N, so there is no bordering.

Readings (the paper states the operator as -1/2 I - D + N without the
normal convention or N for the scalar case):
* nodes, weights and normals as in the Stokes oracle: trapezoid rule in
  the curve parameter, n = (gamma'_y, -gamma'_x)/|gamma'| pointing out of
  Omega;
* with n out of Omega the limit of dn(S mu) from inside Omega is
  (1/2 I + D) mu (the jump relation of the single layer).  The oracle
  and the CUDA path solve (1/2 I + D + N) mu = g, g the flux dn u; the
  paper's -1/2 I - D is the same operator with the opposite sign
  convention for the data;
* N mu = 1 int_Gamma mu dy, rank one.  1/2 I + D has a one-dimensional
  null space, the interior Neumann problem's, since its adjoint 1/2 I + D'
  annihilates constants.  For data with int g = 0 the completed system
  returns int mu = 0 and so solves (1/2 I + D) mu = g exactly;
* diagonal of D: the smooth limit along the curve,
  (gamma''.n) / (4 pi |gamma'|^2), times the node's weight.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .stokes import Geom, quadrature  # noqa: F401  (same discretisation)


def d_entries(g: Geom, rows, cols):
    """D[i, j] w_j for target nodes ``rows`` and source nodes ``cols``; the
    entry with i == j is the smooth diagonal limit."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    rx = g.x[rows][:, None] - g.x[cols][None, :]
    ry = g.y[rows][:, None] - g.y[cols][None, :]
    r2 = rx * rx + ry * ry
    same = rows[:, None] == cols[None, :]
    r2s = np.where(same, 1.0, r2)
    rn = rx * g.nx[rows][:, None] + ry * g.ny[rows][:, None]
    k = -rn / (2.0 * np.pi * r2s)
    k = np.where(same, g.kap[rows][:, None] / (4.0 * np.pi), k)
    return k * g.w[cols][None, :]


def a_entries(g: Geom, rows, cols):
    """Entries of the completed operator 1/2 I + D + N (N = 1 w^T)."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    a = d_entries(g, rows, cols) + g.w[cols][None, :]
    a += 0.5 * (rows[:, None] == cols[None, :])
    return a


def dense_system(g: Geom):
    idx = np.arange(g.N)
    return a_entries(g, idx, idx)


def dense_solve(g: Geom, f, adjoint=False):
    """mu = A^{-1} f (or A^{-T} f) by LU with partial pivoting (library
    routine as the step)."""
    lu = sla.lu_factor(dense_system(g))
    return sla.lu_solve(lu, f, trans=1 if adjoint else 0)


def single_layer(g: Geom, mu, tx, ty):
    """u = S mu at interior targets: -(1/2 pi) sum_j log|t - x_j| mu_j w_j,
    for mu of shape (N,) or (N, nrhs)."""
    tx = np.asarray(tx, float)
    ty = np.asarray(ty, float)
    r = np.hypot(tx[:, None] - g.x[None, :], ty[:, None] - g.y[None, :])
    return -(np.log(r) * g.w[None, :]) @ np.asarray(mu) / (2.0 * np.pi)


def source_potential(tx, ty, src_xy, q):
    """Harmonic test field u = sum_k q_k log|x - s_k| (src_xy (ns, 2),
    q (ns,)); harmonic in Omega when no s_k lies in it."""
    tx = np.asarray(tx, float)
    ty = np.asarray(ty, float)
    u = np.zeros_like(tx)
    for (sx, sy), qk in zip(np.asarray(src_xy), np.asarray(q)):
        u += qk * np.log(np.hypot(tx - sx, ty - sy))
    return u


def source_flux(g: Geom, src_xy, q):
    """dn u on Gamma for u = sum_k q_k log|x - s_k|:
    sum_k q_k (x - s_k).n / |x - s_k|^2."""
    f = np.zeros(g.N)
    for (sx, sy), qk in zip(np.asarray(src_xy), np.asarray(q)):
        rx, ry = g.x - sx, g.y - sy
        f += qk * (rx * g.nx + ry * g.ny) / (rx * rx + ry * ry)
    return f
