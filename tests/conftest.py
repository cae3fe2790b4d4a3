import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libsvt")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_c1_run():
    """The oracle's full solve of the 200 x 200 rank-5 plain FP64 case (seed 0), computed once."""
    from oracle import svt as osvt
    from svt_inputs import config_problem
    p = config_problem("plain_fp64_200", 0)
    res = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default())
    return p, res


@pytest.fixture(scope="session")
def cuda():
    """Builds libsvt (if needed) and returns torch with cuda:0 selected."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_0810_3286_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch
