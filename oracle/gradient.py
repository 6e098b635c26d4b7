"""Shape derivatives for the differentiation path (test infrastructure only,
like the rest of ``oracle``).

The bordered system of Eq. (backwardeq) depends on the curve samples of
every node (position gamma, gamma', gamma'') and on the hole centres c_i.
For an objective of the interior velocity (Eq. completed), the adjoint
method gives its total derivative from two pieces written out here in
plain numpy:

* ``bilinear_grad``: the derivative of L = z^T A(geom) s with respect to
  the samples and centres, for fixed vectors z and s;
* ``energy_grad``: for J = sum_t |u(x_t)|^2 with u = E(geom) s, the
  derivative with respect to s (E^T 2u) and to the samples at fixed s.

Then s = A^{-1} b, A^T z = dJ/ds and dJ/dgeom = dJ/dgeom|_s - dL/dgeom
(``shape_gradient``; the boundary data b must not depend on the varied
samples, as with no-slip holes and a fixed outer curve).  The formulas
follow from differentiating the discretisation's entries (stresslet of
Eq. stokesbie with w = |gamma'| dt and n = (gamma'_y, -gamma'_x)/|gamma'|,
its diagonal limit (gamma''.n)/(2 pi |gamma'|^2) t t^T w, the rank-one N of
Eq. null-spaceop, the Stokeslet/rotlet columns H and the Psi rows of
Sec. 3.1); the CPU tests pin them against central finite differences of
the dense matrix.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from .stokes import dense_system, quadrature, stokeslet_blocks, \
    rotlet_vectors, dl_blocks

FIELDS = ("x", "y", "dx", "dy", "ddx", "ddy")


def samples(x, y, dx, dy, ddx, ddy, dt, comp, centers):
    """A workload-like record of raw curve samples."""
    return SimpleNamespace(x=np.asarray(x, float), y=np.asarray(y, float),
                           dx=np.asarray(dx, float), dy=np.asarray(dy, float),
                           ddx=np.asarray(ddx, float),
                           ddy=np.asarray(ddy, float),
                           dt=np.asarray(dt, float), comp=np.asarray(comp),
                           centers=np.asarray(centers, float))


def bilinear(sm, z, s):
    """L = z^T A s with the dense bordered matrix of the samples sm."""
    return float(np.asarray(z) @ (dense_system(quadrature(sm)) @ s))


def _pair_terms(tx, ty, sx, sy, snx, sny, q, zt):
    """For every target t and source j (arrays broadcast (T, S)):
    F = (1/pi) (r.n_j)(r.q_j)(r.z_t) / |r|^4 with r = x_t - x_j, and its
    derivatives with respect to r, n_j and q_j."""
    rx = tx[:, None] - sx[None, :]
    ry = ty[:, None] - sy[None, :]
    rho = rx * rx + ry * ry
    a = rx * snx[None, :] + ry * sny[None, :]
    b = rx * q[None, :, 0] + ry * q[None, :, 1]
    c = rx * zt[:, None, 0] + ry * zt[:, None, 1]
    with np.errstate(divide="ignore", invalid="ignore"):  # self pairs: caller
        i2 = 1.0 / (np.pi * rho * rho)
        dr_x = (snx[None, :] * b * c + q[None, :, 0] * a * c
                + zt[:, None, 0] * a * b) * i2 - 4.0 * a * b * c * rx * i2 / rho
        dr_y = (sny[None, :] * b * c + q[None, :, 1] * a * c
                + zt[:, None, 1] * a * b) * i2 - 4.0 * a * b * c * ry * i2 / rho
        dn = (rx * b * c * i2, ry * b * c * i2)
        dq = (rx * a * c * i2, ry * a * c * i2)
    return (dr_x, dr_y), dn, dq


def _point_terms(px, py, cx, cy, zt, alpha, beta):
    """d/dr of z.S(r)alpha + z.R(r)beta at r = p - c (Stokeslet
    (1/4pi)(-ln|r| I + r r^T/|r|^2), rotlet r_perp/(4 pi |r|^2)), for points
    (P,) and one centre; returns (P, 2)."""
    rx, ry = px - cx, py - cy
    rho = rx * rx + ry * ry
    za = zt[:, 0] * alpha[0] + zt[:, 1] * alpha[1]
    zr = zt[:, 0] * rx + zt[:, 1] * ry
    ra = rx * alpha[0] + ry * alpha[1]
    f = 1.0 / (4.0 * np.pi)
    gx = f * (-za * rx / rho + (zt[:, 0] * ra + alpha[0] * zr) / rho
              - 2.0 * zr * ra * rx / rho ** 2)
    gy = f * (-za * ry / rho + (zt[:, 1] * ra + alpha[1] * zr) / rho
              - 2.0 * zr * ra * ry / rho ** 2)
    zp = zt[:, 1] * rx - zt[:, 0] * ry            # z . r_perp
    gx += f * beta * (zt[:, 1] / rho - 2.0 * zp * rx / rho ** 2)
    gy += f * beta * (-zt[:, 0] / rho - 2.0 * zp * ry / rho ** 2)
    return np.stack([gx, gy], axis=1)


def _to_samples(sm, gP, gn, gw, gG1, gG2):
    """Chain the per-node derivatives with respect to position, normal,
    weight (and the direct gamma', gamma'' terms) to the samples."""
    G1x, G1y = sm.dx, sm.dy
    sp = np.hypot(G1x, G1y)
    nx, ny = G1y / sp, -G1x / sp
    tx, ty = G1x / sp, G1y / sp
    gnn = gn[:, 0] * nx + gn[:, 1] * ny
    # n = J t, t = gamma'/|gamma'|, J = [[0, 1], [-1, 0]]:
    # dL/dgamma' = (J^T dL/dn - t (n . dL/dn)) / |gamma'|
    gG1x = gG1[:, 0] + (-gn[:, 1] - tx * gnn) / sp + gw * sm.dt * tx
    gG1y = gG1[:, 1] + (gn[:, 0] - ty * gnn) / sp + gw * sm.dt * ty
    return {"x": gP[:, 0], "y": gP[:, 1], "dx": gG1x, "dy": gG1y,
            "ddx": gG2[:, 0], "ddy": gG2[:, 1]}


def bilinear_grad(sm, z, s):
    """dL/d(samples) and dL/d(centres) for L = z^T A(samples) s."""
    g = quadrature(sm)
    N, p = g.N, g.p
    z = np.asarray(z, float)
    s = np.asarray(s, float)
    zm, zl = z[:2 * N].reshape(N, 2), z[2 * N:]
    mu, lam = s[:2 * N].reshape(N, 2), s[2 * N:]
    q = g.w[:, None] * mu
    gP = np.zeros((N, 2))
    gn = np.zeros((N, 2))
    gw = np.zeros(N)
    # off-diagonal stresslet pairs, target i, source j (i != j)
    for i0 in range(0, N, 256):
        i1 = min(N, i0 + 256)
        (dx_, dy_), dn, dq = _pair_terms(g.x[i0:i1], g.y[i0:i1], g.x, g.y,
                                         g.nx, g.ny, q, zm[i0:i1])
        ii = np.arange(i0, i1)
        for arr in (dx_, dy_, dn[0], dn[1], dq[0], dq[1]):
            arr[ii - i0, ii] = 0.0
        gP[i0:i1, 0] += dx_.sum(1)
        gP[i0:i1, 1] += dy_.sum(1)
        gP[:, 0] -= dx_.sum(0)
        gP[:, 1] -= dy_.sum(0)
        gn[:, 0] += dn[0].sum(0)
        gn[:, 1] += dn[1].sum(0)
        gw += dq[0].sum(0) * mu[:, 0] + dq[1].sum(0) * mu[:, 1]
    # diagonal limit: -(dt/2pi) cross (z.g1)(mu.g1)/|g1|^4
    G1 = np.stack([sm.dx, sm.dy], 1)
    G2 = np.stack([sm.ddx, sm.ddy], 1)
    cr = G1[:, 0] * G2[:, 1] - G1[:, 1] * G2[:, 0]
    A = (zm * G1).sum(1)
    B = (mu * G1).sum(1)
    g2 = (G1 * G1).sum(1)
    k = (-sm.dt / (2.0 * np.pi))[:, None]
    dcr1 = np.stack([G2[:, 1], -G2[:, 0]], 1)
    gG1 = k * (dcr1 * (A * B / g2 ** 2)[:, None]
               + cr[:, None] * (zm * B[:, None] + mu * A[:, None])
               / (g2 ** 2)[:, None]
               - 4.0 * (cr * A * B / g2 ** 3)[:, None] * G1)
    gG2 = k * np.stack([-G1[:, 1], G1[:, 0]], 1) * (A * B / g2 ** 2)[:, None]
    # rank-one N: (sum_i z_i.n_i)(sum_j w_j n_j.mu_j)
    Zn = (zm[:, 0] * g.nx + zm[:, 1] * g.ny).sum()
    Sn = (g.w * (g.nx * mu[:, 0] + g.ny * mu[:, 1])).sum()
    gn += zm * Sn + Zn * q
    gw += Zn * (g.nx * mu[:, 0] + g.ny * mu[:, 1])
    # H lambda (Stokeslet / rotlet at the centres) and Psi^T mu rows
    gc = np.zeros((p, 2))
    for c in range(p):
        al = lam[3 * c:3 * c + 2]
        be = lam[3 * c + 2]
        d = _point_terms(g.x, g.y, g.centers[c, 0], g.centers[c, 1], zm, al,
                         be)
        gP += d
        gc[c] -= d.sum(0)
        on = g.comp == c + 1
        zc = zl[3 * c:3 * c + 3]
        perp = -g.y * mu[:, 0] + g.x * mu[:, 1]
        gw += np.where(on, zc[0] * mu[:, 0] + zc[1] * mu[:, 1] + zc[2] * perp,
                       0.0)
        gP[:, 0] += np.where(on, g.w * zc[2] * mu[:, 1], 0.0)
        gP[:, 1] += np.where(on, -g.w * zc[2] * mu[:, 0], 0.0)
    return _to_samples(sm, gP, gn, gw, gG1, gG2), gc


def velocity(sm, s, tx, ty):
    """u = E s at interior points (Eq. completed), (nt, 2)."""
    g = quadrature(sm)
    N = g.N
    mu = np.asarray(s[:2 * N]).reshape(N, 2)
    lam = np.asarray(s[2 * N:])
    D = dl_blocks(tx, ty, g.x, g.y, g.nx, g.ny, g.w)      # (T, N, 2, 2)
    u = np.einsum("tjab,jb->ta", D, mu)
    for c in range(g.p):
        S = stokeslet_blocks(tx, ty, g.centers[c:c + 1, 0],
                             g.centers[c:c + 1, 1])[:, 0]
        R = rotlet_vectors(tx, ty, g.centers[c:c + 1, 0],
                           g.centers[c:c + 1, 1])[:, 0]
        u += np.einsum("tab,b->ta", S, lam[3 * c:3 * c + 2]) + \
            R * lam[3 * c + 2]
    return u


def energy_grad(sm, s, tx, ty):
    """J = sum_t |u_t|^2: returns J, dJ/ds and dJ/d(samples), dJ/d(centres)
    at fixed s."""
    g = quadrature(sm)
    N, p = g.N, g.p
    mu = np.asarray(s[:2 * N]).reshape(N, 2)
    lam = np.asarray(s[2 * N:])
    u = velocity(sm, s, tx, ty)
    ub = 2.0 * u
    q = g.w[:, None] * mu
    (dx_, dy_), dn, dq = _pair_terms(tx, ty, g.x, g.y, g.nx, g.ny, q, ub)
    gP = np.stack([-dx_.sum(0), -dy_.sum(0)], 1)
    gn = np.stack([dn[0].sum(0), dn[1].sum(0)], 1)
    gqx, gqy = dq[0].sum(0), dq[1].sum(0)
    gw = gqx * mu[:, 0] + gqy * mu[:, 1]
    gs = np.zeros(2 * N + 3 * p)
    gs[0:2 * N:2] = g.w * gqx
    gs[1:2 * N:2] = g.w * gqy
    gc = np.zeros((p, 2))
    for c in range(p):
        S = stokeslet_blocks(tx, ty, g.centers[c:c + 1, 0],
                             g.centers[c:c + 1, 1])[:, 0]
        R = rotlet_vectors(tx, ty, g.centers[c:c + 1, 0],
                           g.centers[c:c + 1, 1])[:, 0]
        gs[2 * N + 3 * c:2 * N + 3 * c + 2] = np.einsum("tab,ta->b", S, ub)
        gs[2 * N + 3 * c + 2] = (R * ub).sum()
        d = _point_terms(tx, ty, g.centers[c, 0], g.centers[c, 1], ub,
                         lam[3 * c:3 * c + 2], lam[3 * c + 2])
        gc[c] -= d.sum(0)
    zero = np.zeros((N, 2))
    return float((u * u).sum()), gs, \
        _to_samples(sm, gP, gn, gw, zero, zero), gc


def shape_gradient(sm, b, tx, ty):
    """J(samples) = sum_t |u_t|^2 for the dense solution s = A^{-1} b, and
    dJ/d(samples), dJ/d(centres) by the adjoint method."""
    A = dense_system(quadrature(sm))
    s = np.linalg.solve(A, b)
    J, gs, ge, gce = energy_grad(sm, s, tx, ty)
    z = np.linalg.solve(A.T, gs)
    gb, gcb = bilinear_grad(sm, z, s)
    return J, {f: ge[f] - gb[f] for f in FIELDS}, gce - gcb
