"""O-1: the exact discrete bordered Stokes system, FP64, dense.  Test
infrastructure only (see the package docstring).

Notation follows the paper's Sec. 3.1: boundary Gamma = Gamma_0 u ... u
Gamma_p, density mu (two components per node, interleaved: DOF 2j+a is
component a of node j), lambda = [alpha; beta] ordered hole-major
(alpha_i1, alpha_i2, beta_i).

Discretisation readings (the paper uses a non-uniform trapezoid rule on
spline curves, Sec. 4 opening; it does not give the singular diagonal):
* weights w_j = |gamma'(t_j)| dt_j (trapezoid rule in the curve parameter);
* normal n = (gamma'_y, -gamma'_x)/|gamma'|, which points out of Omega with
  Gamma_0 counter-clockwise and holes clockwise;
* diagonal of the stresslet kernel: its smooth limit as y -> x along the
  curve, (gamma''.n)/(2 pi |gamma'|^2) t t^T with t the unit tangent.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class Geom:
    x: np.ndarray
    y: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    w: np.ndarray
    kap: np.ndarray      # (gamma''.n)/|gamma'|^2
    comp: np.ndarray
    centers: np.ndarray  # (p,2)

    @property
    def N(self):
        return self.x.shape[0]

    @property
    def p(self):
        return self.centers.shape[0]


def quadrature(wl) -> Geom:
    """Trapezoid-rule nodes, weights, normals and the diagonal curvature term
    from curve samples (Sec. 4 opening: trapezoid quadrature in the curve
    parameter; Eq. (stokesbie) needs n(y))."""
    speed = np.hypot(wl.dx, wl.dy)
    nx = wl.dy / speed
    ny = -wl.dx / speed
    w = speed * wl.dt
    kap = (wl.ddx * nx + wl.ddy * ny) / (speed * speed)
    return Geom(np.asarray(wl.x, float), np.asarray(wl.y, float), nx, ny, w,
                kap, np.asarray(wl.comp), np.asarray(wl.centers, float))


def dl_blocks(tx, ty, sx, sy, snx, sny, sw):
    """Stresslet (double-layer) kernel of Eq. (stokesbie) times the source
    weight: D(t,s) w_s = (1/pi) ((t-s).n_s) (t-s)(t-s)^T / |t-s|^4 w_s.
    Returns shape (nt, ns, 2, 2).  Targets and sources must be distinct."""
    rx = np.subtract.outer(tx, sx)
    ry = np.subtract.outer(ty, sy)
    r2 = rx * rx + ry * ry
    rn = rx * snx[None, :] + ry * sny[None, :]
    c = rn / (np.pi * r2 * r2) * sw[None, :]
    out = np.empty(rx.shape + (2, 2))
    out[..., 0, 0] = c * rx * rx
    out[..., 0, 1] = c * rx * ry
    out[..., 1, 0] = c * ry * rx
    out[..., 1, 1] = c * ry * ry
    return out


def stokeslet_blocks(tx, ty, sx, sy):
    """Stokeslet of Sec. 3.1: S(x,c) = (1/4pi)(ln(1/|r|) I + r r^T/|r|^2),
    r = x - c.  Shape (nt, ns, 2, 2)."""
    rx = np.subtract.outer(tx, sx)
    ry = np.subtract.outer(ty, sy)
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    out = np.empty(rx.shape + (2, 2))
    out[..., 0, 0] = (lg + rx * rx / r2) / (4 * np.pi)
    out[..., 0, 1] = (rx * ry / r2) / (4 * np.pi)
    out[..., 1, 0] = out[..., 0, 1]
    out[..., 1, 1] = (lg + ry * ry / r2) / (4 * np.pi)
    return out


def rotlet_vectors(tx, ty, sx, sy):
    """Rotlet of Sec. 3.1: R(x,c) = r^perp / (4 pi |r|^2), r = x - c,
    r^perp = (-r_y, r_x).  Shape (nt, ns, 2)."""
    rx = np.subtract.outer(tx, sx)
    ry = np.subtract.outer(ty, sy)
    r2 = rx * rx + ry * ry
    return np.stack([-ry / (4 * np.pi * r2), rx / (4 * np.pi * r2)], axis=-1)


def _k_node_blocks(g: Geom, ti, sj):
    """2x2 blocks K[ti, sj] of the discretised double-layer operator,
    including the smooth diagonal limit where ti == sj."""
    ti = np.asarray(ti)
    sj = np.asarray(sj)
    same = ti[:, None] == sj[None, :]
    tx, ty = g.x[ti], g.y[ti]
    sx, sy = g.x[sj], g.y[sj]
    with np.errstate(divide="ignore", invalid="ignore"):
        blk = dl_blocks(tx, ty, sx, sy, g.nx[sj], g.ny[sj], g.w[sj])
    if np.any(same):
        a, b = np.nonzero(same)
        j = sj[b]
        tvx, tvy = -g.ny[j], g.nx[j]          # unit tangent
        c = g.kap[j] / (2 * np.pi) * g.w[j]
        blk[a, b, 0, 0] = c * tvx * tvx
        blk[a, b, 0, 1] = c * tvx * tvy
        blk[a, b, 1, 0] = c * tvy * tvx
        blk[a, b, 1, 1] = c * tvy * tvy
    return blk


def k_entries(g: Geom, row_dofs, col_dofs):
    """Entries of the discretised double-layer operator K (Eq. stokesbie,
    trapezoid rule) for DOF lists (DOF 2j+a = component a of node j)."""
    row_dofs = np.asarray(row_dofs, dtype=np.int64)
    col_dofs = np.asarray(col_dofs, dtype=np.int64)
    blk = _k_node_blocks(g, row_dofs // 2, col_dofs // 2)
    ra = (row_dofs % 2)[:, None]
    cb = (col_dofs % 2)[None, :]
    ii = np.arange(len(row_dofs))[:, None]
    jj = np.arange(len(col_dofs))[None, :]
    return blk[ii, jj, ra, cb]


def a11_entries(g: Geom, row_dofs, col_dofs):
    """Entries of -1/2 I + D + N (Eq. completedback): the jump term on equal
    DOFs, the double-layer K, and the null-space completion
    (N mu)(x) = n(x) int n(y).mu(y) dy of Eq. (null-spaceop)."""
    row_dofs = np.asarray(row_dofs, dtype=np.int64)
    col_dofs = np.asarray(col_dofs, dtype=np.int64)
    out = k_entries(g, row_dofs, col_dofs)
    rn = np.where(row_dofs % 2 == 0, g.nx[row_dofs // 2], g.ny[row_dofs // 2])
    cj = col_dofs // 2
    cn = np.where(col_dofs % 2 == 0, g.nx[cj], g.ny[cj]) * g.w[cj]
    out += np.outer(rn, cn)
    out[row_dofs[:, None] == col_dofs[None, :]] -= 0.5
    return out


def h_columns(g: Geom, row_dofs):
    """Rows of H = [S R] (Eq. forwardeq, Sec. 3.1): column 3i+a for hole i is
    the Stokeslet at c_i with unit force e_a (a = 0, 1) and column 3i+2 the
    rotlet of unit torque at c_i."""
    row_dofs = np.asarray(row_dofs, dtype=np.int64)
    nodes = row_dofs // 2
    comp = row_dofs % 2
    p = g.p
    out = np.zeros((len(row_dofs), 3 * p))
    if p == 0:
        return out
    S = stokeslet_blocks(g.x[nodes], g.y[nodes], g.centers[:, 0],
                         g.centers[:, 1])
    R = rotlet_vectors(g.x[nodes], g.y[nodes], g.centers[:, 0],
                       g.centers[:, 1])
    ii = np.arange(len(row_dofs))
    for i in range(p):
        out[:, 3 * i + 0] = S[ii, i, comp, 0]
        out[:, 3 * i + 1] = S[ii, i, comp, 1]
        out[:, 3 * i + 2] = R[ii, i, comp]
    return out


def psi_columns(g: Geom, row_dofs):
    """Rows of the weighted null-space basis: (Psi^T mu) is the integral
    int_{Gamma_i} psi_i^(a) . mu with psi^(1) = e_1, psi^(2) = e_2 and
    psi^(3) = x^perp = (-x_y, x_x) on Gamma_i (Eq. null-space), so the matrix
    entry for DOF (j, c) and column 3i+a is w_j psi_i^(a)(x_j)_c."""
    row_dofs = np.asarray(row_dofs, dtype=np.int64)
    nodes = row_dofs // 2
    comp = row_dofs % 2
    out = np.zeros((len(row_dofs), 3 * g.p))
    for i in range(g.p):
        on = g.comp[nodes] == i + 1
        wj = g.w[nodes]
        out[:, 3 * i + 0] = np.where(on & (comp == 0), wj, 0.0)
        out[:, 3 * i + 1] = np.where(on & (comp == 1), wj, 0.0)
        perp = np.where(comp == 0, -g.y[nodes], g.x[nodes])
        out[:, 3 * i + 2] = np.where(on, wj * perp, 0.0)
    return out


def dense_system(g: Geom):
    """The bordered matrix of Eq. (backwardeq):
    [[-1/2 I + D + N, H], [Psi^T, -I]], size 2N + 3p."""
    n2 = 2 * g.N
    dofs = np.arange(n2)
    A = np.zeros((n2 + 3 * g.p, n2 + 3 * g.p))
    A[:n2, :n2] = a11_entries(g, dofs, dofs)
    A[:n2, n2:] = h_columns(g, dofs)
    A[n2:, :n2] = psi_columns(g, dofs).T
    A[n2:, n2:] = -np.eye(3 * g.p)
    return A


def dense_solve(g: Geom, f, adjoint=False):
    """[mu; lambda] = A^{-1} f (or A^{-T} f) by LU with partial pivoting
    (library routine as the step)."""
    A = dense_system(g)
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, f, trans=1 if adjoint else 0)


def dense_matvec_rows(g: Geom, sol, rows):
    """Rows ``rows`` of A [mu; lambda] for the bordered matrix, computed one
    block row at a time (O(N) per row) for residual spot checks at sizes
    where A cannot be formed."""
    rows = np.asarray(rows, dtype=np.int64)
    n2 = 2 * g.N
    sol = np.asarray(sol)
    if sol.ndim == 1:
        sol = sol[:, None]
    out = np.zeros((len(rows), sol.shape[1]))
    dofs = np.arange(n2)
    for t, r in enumerate(rows):
        if r < n2:
            arow = a11_entries(g, [r], dofs)[0]
            hrow = h_columns(g, [r])[0]
            out[t] = arow @ sol[:n2] + hrow @ sol[n2:]
        else:
            prow = psi_columns(g, dofs)[:, r - n2]
            out[t] = prow @ sol[:n2] - sol[r]
    return out


def point_force_velocity(tx, ty, src_xy, src_f):
    """Velocity of point forces (Stokeslets, Sec. 3.1) at targets:
    u(x) = sum_s S(x, s) f_s.  Returns (nt, 2)."""
    S = stokeslet_blocks(np.asarray(tx), np.asarray(ty), src_xy[:, 0],
                         src_xy[:, 1])
    return np.einsum("tsab,sb->ta", S, src_f)


def boundary_data(g: Geom, src_xy, src_f, holes_zero=False):
    """Right-hand side [f; 0] of Eq. (backwardeq) for boundary data given by
    point forces; ``src_xy``/``src_f`` have shape (nrhs, ns, 2).  With
    ``holes_zero`` the data is kept on Gamma_0 only (no-slip holes)."""
    nrhs = src_xy.shape[0]
    out = np.zeros((2 * g.N + 3 * g.p, nrhs))
    for r in range(nrhs):
        u = point_force_velocity(g.x, g.y, src_xy[r], src_f[r])
        if holes_zero:
            u[g.comp != 0] = 0.0
        out[:2 * g.N, r] = u.reshape(-1)
    return out


def interior_velocity(g: Geom, sol, tx, ty):
    """u = D mu + S alpha + R beta at interior targets (Eq. completed /
    forwardeq).  ``sol`` is (2N+3p, nrhs); returns (nt, 2, nrhs)."""
    sol = np.asarray(sol)
    if sol.ndim == 1:
        sol = sol[:, None]
    n2 = 2 * g.N
    tx = np.asarray(tx)
    ty = np.asarray(ty)
    out = np.zeros((len(tx), 2, sol.shape[1]))
    mu = sol[:n2].reshape(g.N, 2, -1)
    for s0 in range(0, len(tx), 256):
        sl = slice(s0, s0 + 256)
        D = dl_blocks(tx[sl], ty[sl], g.x, g.y, g.nx, g.ny, g.w)
        out[sl] += np.einsum("tsab,sbr->tar", D, mu)
        if g.p:
            S = stokeslet_blocks(tx[sl], ty[sl], g.centers[:, 0],
                                 g.centers[:, 1])
            R = rotlet_vectors(tx[sl], ty[sl], g.centers[:, 0],
                               g.centers[:, 1])
            lam = sol[n2:].reshape(g.p, 3, -1)
            out[sl] += np.einsum("tiab,ibr->tar", S, lam[:, :2])
            out[sl] += np.einsum("tia,ir->tar", R, lam[:, 2])
    return out
