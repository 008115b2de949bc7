"""Host logic of the autotuning cache (no GPU): a measured setting is stored under the system's
shape key and re-applied without timing for the next handle of the same shape."""
import json

import numpy as np

from paper_2501_11962_b300 import synth, tune


class FakeEngine:
    def __init__(self, system, n):
        self.system = system
        self.n_beads = {0: n}
        self.precision = 0
        self.applied = None
        self.timed = 0

    def set_tuning(self, c, b):
        self.applied = (c, b)

    def autotune(self, path_id):
        self.timed += 1
        return dict(col_factor=0.85, bin_factor=1.0), 12.5


def test_cache_round_trip(tmp_path):
    sys_, _ = synth.lj_fcc()
    cache = tmp_path / "tune.json"
    e1 = FakeEngine(sys_, 8)
    r1 = tune.autotune(e1, 0, cache=cache)
    assert r1["cached"] is False and e1.timed == 1
    stored = json.loads(cache.read_text())
    assert list(stored.values())[0]["col_factor"] == 0.85
    e2 = FakeEngine(sys_, 8)
    r2 = tune.autotune(e2, 0, cache=cache)
    assert r2["cached"] is True and e2.timed == 0 and e2.applied == (0.85, 1.0)
    e3 = FakeEngine(sys_, 16)                       # other shape: measured again
    tune.autotune(e3, 0, cache=cache)
    assert e3.timed == 1 and len(json.loads(cache.read_text())) == 2
