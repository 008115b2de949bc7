"""mop_step in CUDA-graph mode: one captured MD step of several uneven paths (sort, list, pair
kernels, bonded terms, gradient and integrator, no host synchronisation) replayed n times must
reproduce the eager steps exactly, replays split over several calls must continue the Philox
step counter, and a list that outgrows its capacity during the replays must be recovered from."""
import numpy as np
import pytest

from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu


def make_engine(graph):
    w = workload(4)
    eng = mop.Engine(w.system)
    for p in (0, 1, 2):                  # N = 24, 40, 64
        eng.set_path(p, w.paths[p])
    ga, gb = w.cv_groups
    eng.add_bias(2, 1.0, 1.0, 0.05, groups=(ga, gb))
    eng.set_graph_mode(graph)
    return eng


def test_graph_step_matches_eager_steps():
    eager = make_engine(False)
    graph = make_engine(True)
    eager.step(6, 2e-5, 2.0, seed=9)
    graph.step(4, 2e-5, 2.0, seed=9)
    graph.step(2, 2e-5, 2.0, seed=9)       # same graph, counter continues on the device
    for p in (0, 1, 2):
        a, b = eager.get_path(p), graph.get_path(p)
        assert np.array_equal(a, b), p
        assert eager.kinetic_energy(p) == graph.kinetic_energy(p)
    va, ga = eager.veff_and_grad(-1)
    vb, gb = graph.veff_and_grad(-1)
    assert np.array_equal(va, vb) and np.array_equal(ga, gb)


def test_graph_recaptures_on_new_parameters():
    eng = make_engine(True)
    eng.step(2, 2e-5, 2.0, seed=9)
    x1 = eng.get_path(1)
    eng.step(2, 1e-5, 0.0, seed=9)       # new dt and gamma: a new graph
    x2 = eng.get_path(1)
    assert not np.array_equal(x1, x2)
    assert np.isfinite(x2).all()


def test_graph_replay_recovers_from_list_overflow():
    """Every bead starts at the same relaxed structure, so the lists are sized for beads with no
    spread; 300 steps of 0.2 fs with a 6000 K thermostat then spread the beads and the lists
    outgrow that capacity during the replays.  mop_step must notice, restore the state it held
    before the replays, grow the capacity and run the steps again: the trajectory equals the
    eager one bit for bit, stays finite, and the repeat is counted."""
    import dataclasses
    w = workload(4, relaxed=True)
    base = np.asarray(w.system.extra["base"], np.float32)
    hot = dataclasses.replace(w.system, temperature=6000.0)
    engines = []
    for graph in (False, True):
        eng = mop.Engine(hot)
        for p, n in enumerate((24, 40)):
            eng.set_path(p, np.repeat(base[None], n, axis=0))
        eng.set_graph_mode(graph)
        eng.step(300, 2e-4, 50.0, seed=5)
        engines.append(eng)
    eager, graph = engines
    assert sum(graph.list_overflows(p) for p in (0, 1)) > 0
    for p in (0, 1):
        a, b = eager.get_path(p), graph.get_path(p)
        assert np.isfinite(b).all()
        assert np.array_equal(a, b), p


def test_autotune_keeps_results():
    w = workload(2, n_beads=8)
    eng = mop.Engine(w.system)
    eng.set_path(0, w.paths[0])
    v0, g0 = eng.veff_and_grad(0)
    best, ms = eng.autotune(0)
    assert best["col_factor"] in (0.85, 1.0, 1.2) and best["bin_factor"] in (0.5, 1.0) and ms > 0
    assert eng.tuning() == best
    for c, b in ((0.85, 1.0), (1.2, 0.5)):
        eng.set_tuning(c, b)
        v, g = eng.veff_and_grad(0)
        assert abs(v[0] - v0[0]) / abs(v0[0]) < 1e-6
        assert np.linalg.norm(g - g0) / np.linalg.norm(g0) < 1e-5
