import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into a dict of int lists."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "residual":
                res = {}
                for tok in vals:
                    site, lst = tok.split(":")
                    res[int(site)] = [int(v) for v in lst.split(",")]
                out[key] = res
            else:
                out[key] = [int(v) for v in vals]
    return out


@pytest.fixture(scope="session")
def ctx():
    """One labelling context on cuda:0 for the GPU tests."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test without a CUDA device")
    import paper_1603_08357_gb300 as ccl
    c = ccl.ccl_context_create(0)
    yield c
    ccl.ccl_context_destroy(c)
