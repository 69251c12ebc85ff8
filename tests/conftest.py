import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "timeout(seconds): per-test time limit (pytest-timeout)")


def golden(name):
    """Path of a fixture under tests/golden/."""
    return os.path.join(ROOT, "tests", "golden", name)


def storage_rounded(rest, state, precision):
    """The populations ``state`` as a grid of the given precision holds them
    once set: deviations from the rest state ``rest`` (the oracle's own
    J f^eq(rho0, 0), both (Q, n1, n2) float64) rounded to nearest in the
    storage type -- FP32; FP16 of 4096 times the deviation; BF16 -- and the
    rest state added back in FP64.  The library's own rest reference may
    differ from the oracle's in the last bit, which moves a rounding by at
    most one unit of the storage type."""
    import numpy as np

    d = np.asarray(state, dtype=np.float64) - rest
    p = str(precision).lower()
    if p in ("0", "fp64"):
        return rest + d
    if p in ("1", "fp32"):
        return rest + d.astype(np.float32).astype(np.float64)
    if p in ("2", "fp16"):
        return rest + (d * 4096.0).astype(np.float32).astype(np.float16).astype(np.float64) / 4096.0
    if p in ("3", "bf16"):
        import torch
        t = torch.from_numpy(d.astype(np.float32)).to(torch.bfloat16).to(torch.float64)
        return rest + t.numpy()
    raise ValueError(precision)
