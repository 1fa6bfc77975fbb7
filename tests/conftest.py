import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built libgpbo.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_08131_b300 import build
    build.build()
    from paper_2403_08131_b300 import gpbo
    c = gpbo.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


@pytest.fixture(scope="session")
def full_size(orc):
    """n = 4096, d = 20, M = 2^20: the bench's workload (five-block function, standardised y);
    the oracle fit is done once per session."""
    from paper_2403_08131_b300 import workloads as W
    w = W.config4()
    ys = (w.y - w.y.mean()) / w.y.std()
    _, Lo, ao = orc.gp_fit(w.X, ys, w.lengthscale, 1.0, w.noise_var)
    return w, ys, Lo, ao
