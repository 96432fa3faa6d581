import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads (minutes)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def rpcg():
    """The CUDA library binding, built in-tree if needed."""
    from paper_2005_07282_gb300 import build
    build.build()
    import paper_2005_07282_gb300 as P
    P.lib()
    return P


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def bits(x):
    """int64 view of float64 data (bit-exact comparison, NaN-safe)."""
    import numpy as np
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def pcg_2x2_golden():
    """The hand-worked two-iteration trace of tests/golden/pcg_2x2_trace.txt:
    {loop test l: {name: [values]}}, plus the system it belongs to."""
    trace = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "pcg_2x2_trace.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        l, name, *vals = line.split()
        trace.setdefault(int(l), {})[name] = [float.fromhex(v) for v in vals]
    import numpy as np

    import synth
    A = synth.CSR(2, np.array([0, 2, 4], dtype=np.int32), np.array([0, 1, 0, 1], dtype=np.int32),
                  np.array([4.0, 1.0, 1.0, 3.0]), "spd2x2")
    return A, np.array([3.0, 0.5]), trace
