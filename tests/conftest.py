import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


@pytest.fixture(scope="session")
def oracle():
    import oracle as o
    o.build()
    return o


@pytest.fixture(scope="session")
def svlib():
    """Built libsv.so + the binding module (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2106_13995_gb300 as P
    P.build()
    from paper_2106_13995_gb300 import sim
    return sim


def fidelity_metrics(ref, got):
    """(1 - F, max |amplitude error|) of a GPU state against an oracle state."""
    import numpy as np
    import oracle as o
    return o.infidelity(ref, got), float(np.max(np.abs(np.asarray(got, dtype=np.complex128) - ref)))
