"""Runtime pieces around the method: the device allocation cache and the
measured arithmetic peaks used as roofline denominators."""
import numpy as np
import pytest

import workloads as W
from gpu_util import solver

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_measured():
    import paper_2001_11619_gb300 as skel
    pk = skel.measure_alu_peaks()
    # GB300: FP64 about 1.2 TFLOP/s, FP32 about 70; loose bounds catch a
    # timing or counting error, not a slow clock
    assert 0.2 < pk["fp64_tflops"] < 5.0
    assert 10.0 < pk["fp32_tflops"] < 200.0
    assert pk["fp32_tflops"] > 10 * pk["fp64_tflops"]


def test_cached_blocks_are_reused_and_released():
    """The blocks a closed solver frees stay cached, a second solver on the same geometry
    gives the same bits from reused memory, and releasing the cache leaves
    later solvers working."""
    import paper_2001_11619_gb300 as skel
    wl = W.star1()
    rhs = np.random.default_rng(4).standard_normal(wl.n_unknowns)
    a = solver(wl)
    a.factor()
    xa = a.solve(rhs)
    fac_bytes = a.stats()["fac_bytes"]
    a.close()
    b = solver(wl)
    assert fac_bytes > 0 and b.stats()["cached_device_bytes"] > 0
    b.factor()
    assert np.array_equal(b.solve(rhs), xa)
    b.close()
    skel.release_cached_memory()
    c = solver(wl)
    c.factor()
    assert np.array_equal(c.solve(rhs), xa)
    c.close()
