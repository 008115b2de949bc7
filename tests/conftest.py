import sys
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


_CACHE = {}


RELAXED = ROOT / "tests" / "golden" / "relaxed"


def workload(k, relaxed=False, **kw):
    """Seeded workload k (1..5), cached per test session.  relaxed: around the stored relaxed
    base structure (tests/golden/relax_inputs.py) instead of the generated one."""
    from paper_2501_11962_b300 import synth
    key = (k, relaxed, tuple(sorted(kw.items())))
    if key not in _CACHE:
        base = np.load(RELAXED / f"cfg{k}.npy") if relaxed else None
        _CACHE[key] = synth.config(k, base=base, **kw)
    return _CACHE[key]


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(20250121)
