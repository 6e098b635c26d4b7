"""The C ABI library builds for sm_103a, loads, and exports every entry
point that include/skel.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "skel.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(skel_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("skel_build_tree", "skel_factor", "skel_update_moved_nodes",
              "skel_solve", "skel_solve_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2001_11619_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    for n in _declared():
        assert hasattr(lib, n), n


def test_package_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_2001_11619_gb300 as pkg
    from paper_2001_11619_gb300 import _build
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        pkg.load_library(build_if_missing=False)


def test_errors_without_gpu_are_reported_not_fatal():
    """On a machine without a GPU the library returns an error code; it
    never falls back to the CPU."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2001_11619_gb300 as skel
    import workloads as W
    wl = W.custom([W.circle(1.0)], [64], n_targets=0)
    with pytest.raises(skel.SkelError):
        s = skel.Solver(wl)
        s.factor()


def test_binding_checks_lengths_the_library_reads():
    """The library reads nt entries of tx and of ty and n entries of each
    solution-sized vector; the binding refuses shorter or mismatched
    arrays before any pointer reaches the library."""
    import numpy as np
    import paper_2001_11619_gb300 as skel
    x, y, nt = skel._targets(np.zeros(5), np.ones(5))
    assert nt == 5 and len(y.obj) == 5
    with pytest.raises(ValueError):
        skel._targets(np.zeros(5), np.zeros(4))
    with pytest.raises(ValueError):
        skel._targets(np.zeros((5, 1)), np.zeros((5, 1)))
    assert len(skel._vec(np.zeros(7), 7, "s").obj) == 7
    assert skel._vec(np.zeros((7, 1)), 7, "s").obj.shape == (7,)
    with pytest.raises(ValueError):
        skel._vec(np.zeros(6), 7, "s")
    with pytest.raises(ValueError):
        skel._vec(np.zeros((7, 2)), 7, "s")
