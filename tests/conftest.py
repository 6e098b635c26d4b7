import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: larger CPU case (still minutes at most)")


@pytest.fixture(scope="session")
def star1():
    import workloads
    return workloads.star1()


@pytest.fixture(scope="session")
def star1_dense(star1):
    import oracle
    g = oracle.quadrature(star1)
    f = oracle.boundary_data(g, star1.src_xy, star1.src_f)
    return g, f, oracle.dense_solve(g, f)


@pytest.fixture(scope="session")
def star1_fac(star1):
    import oracle
    return oracle.factor(star1)
