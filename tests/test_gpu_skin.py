"""Verlet skin of the cluster-pair lists (mop_set_list_skin): a list built for rc + skin is kept
while no atom of any bead has moved more than skin / 2, and the results stay those of the oracle
(the pair kernels still test r < rc); a larger move rebuilds it; MD steps with kept lists follow
the steps with rebuilt lists to rounding."""
import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import mop
from tests.conftest import workload
from tests.test_gpu_parity import TOL_F, TOL_H, TOL_V, rel

pytestmark = pytest.mark.gpu


def check_against_oracle(eng, X):
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(eng.system).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"),
                                       hvp_mode=oracle.HVP_ANALYTIC)
    N = X.shape[0]
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1]
    H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(F, r["F"][:N - 1]) < TOL_F
    assert rel(H, r["Heta"][:N - 1]) < TOL_H
    assert rel(G, r["G"]) < TOL_F
    return v, G


def test_kept_list_matches_oracle_and_rebuilds_past_half_the_skin():
    w = workload(2, n_beads=6)
    X = w.paths[0]
    rng = np.random.default_rng(7)
    eng = mop.Engine(w.system)
    eng.set_list_skin(0.05)
    eng.set_path(0, X)
    check_against_oracle(eng, X)
    assert eng.list_stats(0) == (1, 0)
    # every coordinate moved by less than skin / 2 / sqrt(3): the list is kept
    X2 = (X + rng.uniform(-0.014, 0.014, X.shape)).astype(np.float32)
    eng.set_path(0, X2)
    v2, G2 = check_against_oracle(eng, X2)
    assert eng.list_stats(0) == (1, 1)
    # the same positions with a list rebuilt at every evaluation: equal to rounding
    ref = mop.Engine(w.system)
    ref.set_path(0, X2)
    v2r, G2r = ref.veff_and_grad(0)
    assert abs(v2[0] - v2r[0]) / abs(v2r[0]) < 1e-7
    assert rel(G2, G2r) < 1e-6
    # one atom of one bead moves 0.03 nm > skin / 2: rebuilt
    X3 = X2.copy()
    X3[2, 17, 0] += 0.03
    eng.set_path(0, X3)
    check_against_oracle(eng, X3)
    assert eng.list_stats(0) == (2, 1)


def test_md_steps_with_kept_lists_follow_rebuilt_lists():
    w = workload(2, n_beads=4)
    runs = []
    for skin in (0.0, 0.05):
        eng = mop.Engine(w.system)
        eng.set_list_skin(skin)
        eng.set_path(0, w.paths[0])
        eng.step(6, 1e-5, 0.0, 1)
        runs.append((eng.get_path(0).astype(np.float64), eng.kinetic_energy(0), eng.list_stats(0)))
    (x0, ke0, s0), (x1, ke1, s1) = runs
    assert s0[1] == 0 and s1[1] > 0            # the skin run kept its list at least once
    assert np.abs(x1 - x0).max() < 1e-5
    assert ke1 == pytest.approx(ke0, rel=1e-4)


def test_skin_is_validated():
    w = workload(2, n_beads=3)
    eng = mop.Engine(w.system)
    for bad in (-0.1, float("nan"), 0.7):      # box 3.10 nm, rc 0.9 nm: rc + skin must stay below L/2
        with pytest.raises(mop.MopError) as ei:
            eng.set_list_skin(bad)
        assert ei.value.status == mop.MOP_ERR_ARG
