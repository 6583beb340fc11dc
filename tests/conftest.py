import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def ball12_lu():
    """The oracle's 12^3 penetrable ball (k0 = 2, rho = 1.5, c = 0.7, four-point rule) with
    its dense collocation matrix LU-factorised once per session: the Mie-series,
    exterior-field and reciprocity pins all solve this system."""
    import scipy.linalg as sla

    from oracle import vsie_oracle as O
    from paper_2607_06429_b300 import workloads as W
    w = W.single_ball(12, 3, 2.0)
    D = O.Discretisation.from_workload(w)
    return w, D, sla.lu_factor(D.assemble())
