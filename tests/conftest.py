import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def load_golden_matrices(name):
    """Parse a tests/golden fixture: '#' comments, 'matrix NAME ROWS COLS' headers, rows."""
    mats, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("matrix"):
                _, cur, rows, cols = line.split()
                mats[cur] = (int(rows), int(cols), [])
                continue
            mats[cur][2].append([int(v) for v in line.split()])
    out = {}
    for k, (r, c, rows) in mats.items():
        a = np.array(rows, dtype=np.int64)
        assert a.shape == (r, c), (name, k, a.shape)
        out[k] = a
    return out


def load_golden_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, dtype=np.int64)


@pytest.fixture(scope="session")
def cuda_device():
    """The CUDA device for -m gpu tests.  Fails (does not skip) when no GPU is present."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but torch.cuda.is_available() is False")
    return torch.device("cuda:0")
