"""Accuracy against closed forms at full size on the GPU (the paper's
Sec. 4.1 experiments, scaled to 32768 nodes).

Couette flow between concentric circles (constants from
tests/golden/couette.txt, hand-derived there) through the whole path:
factorization, solve, interior velocity.  Checks:
- in the FP64 form the error against the exact flow tracks the ID
  tolerance from 1e-4 to 1e-12 (the paper's error-versus-tolerance test)
  and is below 1e-10 at 1e-12;
- the mixed form at ID tolerance 1e-6 with GMRES refinement reaches the
  same 1e-10."""
import os

import numpy as np
import pytest

import workloads as W
from gpu_util import solver

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def couette_case(n_outer=21846, n_inner=10922):
    """Workload, boundary data (2N+3p), targets and the exact velocity."""
    R1, R2, V1, V2, A, B = np.loadtxt(os.path.join(GOLDEN, "couette.txt"))
    w = W.custom([W.circle(R2), W.circle(R1, ccw=False)], [n_outer, n_inner],
                 n_targets=0, leaf_size=64)
    N = w.N
    f = np.zeros((2 * N + 3, 1))
    outer = np.asarray(w.comp) == 0
    V = np.where(outer, V2, V1)
    r = np.hypot(w.x, w.y)
    f[:2 * N:2, 0] = -V * w.y / r
    f[1:2 * N:2, 0] = V * w.x / r
    rr, tt = np.meshgrid(np.linspace(R1 + 0.05, R2 - 0.05, 19),
                         np.linspace(0, 2 * np.pi, 24, endpoint=False))
    tx, ty = (rr * np.cos(tt)).ravel(), (rr * np.sin(tt)).ravel()
    ut = A * rr.ravel() + B / rr.ravel()
    ue = np.stack([-ut * np.sin(tt.ravel()), ut * np.cos(tt.ravel())], 1)
    return w, f, tx, ty, ue


def _error(s, f, tx, ty, ue):
    u = s.eval_velocity(s.solve(f), tx, ty)[:, :, 0]
    return float(np.abs(u - ue).max() / np.abs(ue).max())


def test_couette_error_tracks_the_id_tolerance():
    w, f, tx, ty, ue = couette_case()
    assert w.N == 32768
    errs = {}
    for tol in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12):
        s = solver(w, id_tol=tol)
        s.factor()
        errs[tol] = _error(s, f, tx, ty, ue)
        s.close()
    print("Couette, 32768 nodes, error by ID tolerance:", errs)
    for tol, e in errs.items():
        assert e < 10 * tol + 1e-12, (tol, e)
    assert errs[1e-12] < 1e-10
    # coarser tolerances give visibly larger errors (the ID error, not
    # the quadrature, dominates above 1e-10)
    assert errs[1e-4] > 10 * errs[1e-8] and errs[1e-6] > 10 * errs[1e-10]


def test_couette_mixed_form():
    import paper_2001_11619_gb300 as skel
    w, f, tx, ty, ue = couette_case()
    s = solver(w, id_tol=1e-6, precision=skel.MIXED, gmres_tol=1e-12,
               gmres_maxit=60)
    s.factor()
    e = _error(s, f, tx, ty, ue)
    st = s.stats()
    s.close()
    print("Couette, 32768 nodes, mixed form:", e, st["gmres_iters"])
    assert e < 1e-10
    assert 0 < st["gmres_iters"] <= 6
