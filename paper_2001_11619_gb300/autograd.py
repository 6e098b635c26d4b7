"""Differentiable objective of the Stokes velocity for torch.

``velocity_energy`` returns J = sum_t |u(x_t)|^2 of the interior velocity
(the solution of the bordered system for point-force boundary data with
no-slip holes) as a torch scalar whose gradient flows to the boundary
samples (x, y, gamma', gamma'' per node) and the hole centres.  The forward
pass factors the geometry, solves and evaluates J (skel_velocity_energy)
and keeps the factorization; the backward pass runs the adjoint part
(skel_velocity_energy_gradient: the velocity derivative, the transposed
factored solve and the derivative of the double-layer matrix) and then
frees it.  An evaluation that is never differentiated (a line-search
trial, say) pays for the value only.  A parametrisation built from torch
operations (for instance the Fourier coefficients of the holes) then
receives dJ/dtheta through torch's chain rule.

The boundary data must not depend on the differentiated samples: the
outer curve, which carries the point-force data, is held fixed, and hole
data are zero (Sec. 4.3's setting of moving interior shapes).
"""
from __future__ import annotations

from types import SimpleNamespace

import torch

from . import GEOM_FIELDS, Solver


class _VelocityEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, dx, dy, ddx, ddy, centers, dt, comp, src_xy,
                src_f, tx, ty, options):
        geom = SimpleNamespace(x=x.detach(), y=y.detach(), dx=dx.detach(),
                               dy=dy.detach(), ddx=ddx.detach(),
                               ddy=ddy.detach(), dt=dt, comp=comp,
                               centers=centers.detach())
        s = Solver(geom, **options)
        try:
            s.factor()
            f = s.point_force_rhs(src_xy, src_f, holes_zero=True, like=x)
            J, sol = s.velocity_energy(f[:, 0], tx, ty)
        except Exception:
            s.close()
            raise
        # the factorization stays for the backward pass
        ctx.solver, ctx.sol, ctx.tx, ctx.ty = s, sol, tx, ty
        return torch.tensor(J, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gJ):
        s = ctx.solver
        try:
            g = s.velocity_energy_gradient_at(ctx.sol, ctx.tx, ctx.ty)
        finally:
            s.close()
            ctx.solver = None
        grads = [gJ * g[k] for k in GEOM_FIELDS] + [gJ * g["centers"]]
        return (*grads, None, None, None, None, None, None, None)


def velocity_energy(x, y, dx, dy, ddx, ddy, centers, dt, comp, src_xy, src_f,
                    tx, ty, **options):
    """J = sum_t |u(tx_t, ty_t)|^2, differentiable with respect to x, y, dx,
    dy, ddx, ddy (node samples) and centers.  ``options`` go to Solver
    (leaf_size, n_proxy, proxy_ratio, id_tol, precision, ...)."""
    return _VelocityEnergy.apply(x, y, dx, dy, ddx, ddy, centers, dt, comp,
                                 src_xy, src_f, tx, ty, options)
