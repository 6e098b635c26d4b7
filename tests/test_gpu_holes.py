"""Hole deletion and insertion through the fast update (Sec. 2.8 marking,
skel_update_geometry): after each change the solve equals that of a fresh
factorization of the new geometry bit for bit (FP64 and mixed forms), only
part of the boxes is recompressed, and the FP64 operator residual stays at
the solver's tolerance."""
import numpy as np
import pytest

import workloads as W
from gpu_util import solver, to_device

pytestmark = pytest.mark.gpu


def _pair(wl, prec):
    import paper_2001_11619_gb300 as skel
    kw = {} if prec == "fp64" else dict(precision=skel.MIXED, id_tol=1e-6,
                                        gmres_tol=1e-13, gmres_maxit=60)
    return solver(wl, **kw)


def _check_against_fresh(s, wl, prec):
    import torch
    f = s.point_force_rhs(wl.src_xy, wl.src_f,
                          like=torch.zeros(1, dtype=torch.float64,
                                           device="cuda"))
    fresh = _pair(wl, prec)
    fresh.factor()
    a, b = s.solve(f), fresh.solve(f)
    assert torch.equal(a, b)
    r = s.matvec(a) - f
    assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) < 1e-10
    assert s.stats()["root_skeleton"] == fresh.stats()["root_skeleton"]
    fresh.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_delete_then_insert_a_hole(prec):
    wl = W.scaled(W.star16(), 8, n_targets=16)
    s = _pair(wl, prec)
    s.factor()
    # delete hole 5: later holes are renumbered, their nodes shift down
    w1, old1 = W.remove_hole(wl, 5)
    s.update_geometry(to_device(w1), old1)
    st = s.stats()
    assert s.N == w1.N and s.p == w1.p == wl.p - 1
    assert 0 < st["last_dirty"] < st["last_boxes"]
    _check_against_fresh(s, w1, prec)
    # insert it again, appended as the last hole
    w2, old2 = W.add_hole(w1, wl.curves[5], wl.counts[5])
    s.update_geometry(to_device(w2), old2)
    st = s.stats()
    assert s.p == wl.p and 0 < st["last_dirty"] < st["last_boxes"]
    _check_against_fresh(s, w2, prec)
    # and a plain move afterwards still matches a fresh factorization
    w3 = W.move_hole(w2, 2, (0.003, -0.002))
    sl = w3.node_slice(2)
    s.update_moved_nodes(np.arange(sl.start, sl.stop), to_device(w3))
    _check_against_fresh(s, w3, prec)
    s.close()


def test_invalid_old_ids_are_rejected():
    import paper_2001_11619_gb300 as skel
    wl = W.scaled(W.star16(), 16, n_targets=4)
    s = solver(wl)
    s.factor()
    w1, old1 = W.remove_hole(wl, 3)
    bad = old1.copy()
    bad[[10, 11]] = bad[[11, 10]]  # not increasing
    with pytest.raises(skel.SkelError):
        s.update_geometry(to_device(w1), bad)
    with pytest.raises(ValueError):
        s.update_geometry(to_device(w1), old1[:-1])
    s.close()
