"""The stored relaxed base structures (tests/golden/relaxed/) are what tests/golden/relax_inputs.py
writes from the seeded generator and the oracle's forces: re-running it for the water box
reproduces the file bit for bit, and every stored structure has a much lower energy than the
generated one it came from."""
import importlib.util
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import synth

GOLD = Path(__file__).resolve().parent / "golden"


def _relax_module():
    spec = importlib.util.spec_from_file_location("relax_inputs", GOLD / "relax_inputs.py")
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_relaxed_water_box_is_reproduced():
    m = _relax_module()
    stored = m.load(2)
    assert stored is not None
    again = m.relax(2)
    assert np.array_equal(again, stored)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_relaxed_structures_lower_the_energy(k):
    m = _relax_module()
    x = m.load(k)
    assert x is not None
    w = synth.config(k, n_beads=1)
    o = oracle.Oracle(w.system)
    _, u0 = o.forces(np.asarray(w.system.extra["base"], np.float64))
    F, u1 = o.forces(x.astype(np.float64))
    assert u0 > 0.0 > u1                   # from strained (U > 0) to bound (U < 0)
    assert np.abs(F).max() < 1e3           # no close contacts left
