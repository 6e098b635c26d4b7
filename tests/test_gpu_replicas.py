"""The replica driver on one GPU: hole-move trials evaluated through
updates of one factorization (moved_hole_objective + run_batch) equal the
same objective from a fresh factorization of every trial geometry, bit
for bit (an update reproduces a fresh factorization, Sec. 2.8)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import solver, to_device

pytestmark = pytest.mark.gpu


def test_hole_move_trials_equal_fresh_factorizations():
    import torch

    from paper_2001_11619_gb300 import replicas as R
    wl = W.scaled(W.star16(), 8, n_targets=64)
    tx = torch.tensor(wl.targets[:, 0].copy(), device="cuda")
    ty = torch.tensor(wl.targets[:, 1].copy(), device="cuda")
    s = solver(wl)
    s.factor()
    ev = R.moved_hole_objective(s, wl, (tx, ty), to_device, W.move_hole)
    trials = [(3, 0.004, -0.002), (3, -0.003, 0.001), (7, 0.002, 0.002),
              (3, 0.0, 0.0)]
    got = R.run_batch(trials, ev)

    def fresh(task):
        h, dx, dy = task
        cur = W.move_hole(wl, h, (dx, dy))
        f = solver(cur)
        f.factor()
        rhs = f.point_force_rhs(cur.src_xy, cur.src_f, like=tx)
        u = f.eval_velocity(f.solve(rhs), tx, ty)
        f.close()
        return float((u.double() ** 2).sum().item())

    want = [fresh(t) for t in trials]
    assert got == want
    # the unmoved trial is the objective of the original geometry
    assert got[3] == fresh((1, 0.0, 0.0))
    s.close()
