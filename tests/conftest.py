import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def headline_oracle():
    """The oracle's build of the 3D 1/r workload at N = 2^20 (about half a
    minute of CPU), shared by the full-size parity tests."""
    import oracle
    import smash_inputs as si
    w = si.make_workload("3d_invr_1m")
    ho = oracle.H2(w["x"], w["kernel"], w["leaf"], w["order"], w["tol"])
    return w, ho, ho.export()


@pytest.fixture(scope="session")
def sphere_oracle():
    """The oracle's build of the sphere Yukawa workload at N = 2^20 (order 5;
    about a minute and a half of CPU), shared by the full-size tests of the
    mixed precisions."""
    import oracle
    import smash_inputs as si
    w = si.make_workload("sphere_yukawa_1m")
    ho = oracle.H2(w["x"], w["kernel"], w["leaf"], w["order"], w["tol"])
    return w, ho, ho.export()
