import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libisg.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def table1_triples():
    """(Nc, M, E) triples of Table 1 (Sec. 4), 4x4 periodic ferromagnet."""
    path = os.path.join(ROOT, "tests", "golden", "table1_4x4_periodic.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                nc, m, e = (int(x) for x in line.split())
                rows.append((nc, m, e))
    return rows


@pytest.fixture(scope="session")
def isg():
    """The native binding, with libisg.so built (build() is a no-op when it is up to date)."""
    from paper_1110_2561_gb300 import build as _build, isg as _isg
    _build.build()
    _isg.lib()
    return _isg


@pytest.fixture(scope="session")
def cuda(isg):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")
