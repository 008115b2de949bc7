"""The instrumentation behind the benchmark's roofline figures: the pair count that is the
numerator of the achieved FLOP/s, the per-pass CUDA-event times that are its denominator, and
the measured FP32 peak quoted beside the nominal one."""
import numpy as np
import pytest

from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu


def brute_force_pairs(system, X, band):
    """Unordered non-excluded atom pairs with minimum-image distance below rc, summed over the beads
    of X, and how many of them lie within `band` nm of rc (where the GPU's FP32 coordinates may
    decide the other way)."""
    Q = system.n_atoms
    iu, ju = np.triu_indices(Q, 1)
    excl = (system.mol_id[iu] == system.mol_id[ju]) & (np.abs(system.mol_local[iu] - system.mol_local[ju]) <= 2)
    keep = ~excl
    iu, ju = iu[keep], ju[keep]
    L = np.asarray(system.box, np.float64)
    inside = edge = 0
    for n in range(X.shape[0]):
        d = X[n, iu] - X[n, ju]
        d -= L * np.round(d / L)
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        inside += int(np.count_nonzero(r < system.rc))
        edge += int(np.count_nonzero(np.abs(r - system.rc) < band))
    return inside, edge


@pytest.mark.parametrize("kernels", ["default", "blhalf"])
def test_count_pairs_matches_brute_force(kernels, monkeypatch):
    if kernels != "default":
        monkeypatch.setenv("MOP_PAIR_KERNELS", kernels)
    w = workload(2, relaxed=True, n_beads=6)
    eng = mop.Engine(w.system)
    eng.set_path(0, w.paths[0])
    eng.veff_and_grad(0)
    unique, listed = eng.count_pairs(0)
    eng.close()
    # beads 1 .. N-1 need forces (bead N needs none, Eq. 7)
    inside, edge = brute_force_pairs(w.system, w.paths[0][:-1].astype(np.float64), 1e-5)
    assert inside > 0
    assert abs(unique - inside) <= edge
    # the list evaluates every counted pair, from both sides on the full list
    assert listed >= (2 if kernels == "default" else 1) * unique


def test_pass_times_cover_the_evaluation():
    w = workload(2, relaxed=True)
    eng = mop.Engine(w.system)
    eng.set_path(0, w.paths[0])
    eng.set_profiling(True)
    eng.veff_and_grad(0)
    eng.veff_and_grad(0)
    p = eng.pass_ms()
    eng.close()
    assert len(p) == 6 and all(v >= 0.0 for v in p.values())
    names = list(p)
    # the pair passes are the largest of the evaluation
    assert p[names[1]] > 0.0 and p[names[3]] > 0.0
    assert p[names[1]] + p[names[3]] > 0.5 * sum(p.values())


def test_measured_fp32_peak_is_plausible():
    t = mop.measure_fp32_peak(0)
    # 148 SMs x 128 lanes x 2 flops x at most 2.032 GHz = 77 TFLOP/s; a dependent-FMA kernel
    # reaches most of it at any clock the part runs at under load
    assert 20.0 < t < 80.0
