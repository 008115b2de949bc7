"""mop_step in CUDA-graph mode: one captured MD step of several uneven paths (sort, list, pair
kernels, bonded terms, gradient and integrator, no host synchronisation) replayed n times must
reproduce the eager steps exactly, and replays split over several calls must continue the
Philox step counter."""
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


def test_graph_replay_reports_list_overflow():
    # from these unrelaxed structures a large step moves atoms far enough that the lists outgrow
    # the capacity sized before the capture; mop_step must say so rather than return bad steps
    eng = make_engine(True)
    with pytest.raises(mop.MopError) as ei:
        for _ in range(20):
            eng.step(5, 5e-4, 2.0, seed=9)
    assert ei.value.status == mop.MOP_ERR_STATE


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
