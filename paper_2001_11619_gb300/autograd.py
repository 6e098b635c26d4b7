"""Differentiable objective of the Stokes velocity for torch.

``velocity_energy`` returns J = sum_t |u(x_t)|^2 of the interior velocity
(the solution of the bordered system for point-force boundary data with
no-slip holes) as a torch scalar whose gradient flows to the boundary
samples (x, y, gamma', gamma'' per node) and the hole centres.  The forward
pass factors the geometry, solves, and forms the adjoint gradient with the
library's shape-derivative kernels (skel_grad_velocity, skel_solve_adjoint,
skel_grad_bilinear); backward scales it.  A parametrisation built from
torch operations (for instance the Fourier coefficients of the holes) then
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
            J, _, grad = s.velocity_energy_gradient(f, tx, ty)
        finally:
            s.close()
        ctx.save_for_backward(*[grad[k] for k in GEOM_FIELDS],
                              grad["centers"])
        return torch.tensor(J, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gJ):
        grads = [gJ * g for g in ctx.saved_tensors]
        return (*grads, None, None, None, None, None, None, None)


def velocity_energy(x, y, dx, dy, ddx, ddy, centers, dt, comp, src_xy, src_f,
                    tx, ty, **options):
    """J = sum_t |u(tx_t, ty_t)|^2, differentiable with respect to x, y, dx,
    dy, ddx, ddy (node samples) and centers.  ``options`` go to Solver
    (leaf_size, n_proxy, proxy_ratio, id_tol, precision, ...)."""
    return _VelocityEnergy.apply(x, y, dx, dy, ddx, ddy, centers, dt, comp,
                                 src_xy, src_f, tx, ty, options)
