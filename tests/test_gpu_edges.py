"""Edge cases of the batch: a 13-atom system (one ragged cluster, molecules with bonds and
angles, mixed precision, FP64 and SPME) against the oracle, and the largest batch, 64 paths
evaluated in one call, against the same paths one call each."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import mop, synth
from tests.conftest import workload
from tests.test_gpu_parity import TOL_F, TOL_H, TOL_V, rel

pytestmark = pytest.mark.gpu


def tiny_system(seed=5, box=(2.4, 2.4, 2.4)):
    """13 atoms in a small box: two bent 3-atom molecules and 7 single atoms, 2 LJ types,
    charges summing to zero, no two atoms closer than 0.25 nm (nearest image)."""
    rng = np.random.default_rng(seed)
    box = np.array(box, dtype=np.float64)
    pos = []
    for m in range(2):                              # molecules: bond 0.15 nm, angle ~109.5 deg
        while True:
            c = rng.random(3) * box
            d1 = rng.normal(size=3)
            d1 /= np.linalg.norm(d1)
            d2 = rng.normal(size=3)
            d2 -= d2 @ d1 * d1
            d2 /= np.linalg.norm(d2)
            th = np.deg2rad(109.5)
            cand = [c, c + 0.15 * d1, c + 0.15 * (np.cos(th) * d1 + np.sin(th) * d2)]
            if all(np.linalg.norm((p - q + box / 2) % box - box / 2) > 0.25 for p in pos for q in cand):
                pos += cand
                break
    while len(pos) < 13:
        q = rng.random(3) * box
        if all(np.linalg.norm((p - q + box / 2) % box - box / 2) > 0.25 for p in pos):
            pos.append(q)
    pos = np.array(pos)
    Q = len(pos)
    charge = rng.uniform(-0.5, 0.5, Q)
    charge -= charge.mean()
    sys = synth.System(
        box=box, type=np.array([0, 1, 1] * 2 + [0, 1] * 3 + [0], np.int32),
        lj_sigma=np.array([0.32, 0.25]), lj_eps=np.array([0.65, 0.3]), charge=charge,
        mass=np.array([16.0, 1.0, 1.0] * 2 + [12.0, 14.0] * 3 + [23.0]),
        mol_id=np.array([0, 0, 0, 1, 1, 1] + list(range(2, 9)), np.int32),
        mol_local=np.array([0, 1, 2, 0, 1, 2] + [0] * 7, np.int32),
        bond_ij=np.array([[0, 1], [0, 2], [3, 4], [3, 5]], np.int32), bond_r0=np.full(4, 0.15),
        bond_k=np.full(4, 3.0e5), angle_ijk=np.array([[1, 0, 2], [4, 3, 5]], np.int32),
        angle_th0=np.full(2, np.deg2rad(109.5)), angle_k=np.full(2, 400.0), rc=1.0)
    return sys, pos


def tiny_path(pos, N=5, seed=9):
    rng = np.random.default_rng(seed)
    return (pos[None] + rng.normal(0.0, 0.01, (N,) + pos.shape)).astype(np.float32)


@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_tiny_ragged_system_matches_oracle(prec):
    sys, pos = tiny_system()
    X = tiny_path(pos)
    eng = mop.Engine(sys, precision=prec)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"), hvp_mode=oracle.HVP_ANALYTIC)
    N = X.shape[0]
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1]
    H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
    tol = 1e-8 if prec == mop.MOP_PREC_FP64 else 1.0   # FP64: every quantity within ~1e-13
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V * tol
    assert rel(F, r["F"][:N - 1]) < TOL_F * tol
    assert rel(H, r["Heta"][:N - 1]) < TOL_H * tol
    assert rel(G, r["G"]) < TOL_F * tol


@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_potential_shift_cutoff_matches_oracle(prec):
    """The potential-shift modifier (phi(r) - phi(rc), force cut at rc) instead of the shifted
    force.  On this 13-atom system no pair lies within FP32 rounding of rc, so both precisions
    take the same in/out decision per pair as the oracle."""
    sys, pos = tiny_system()
    sys = dataclasses.replace(sys, cutoff_mode=synth.CUTOFF_POT_SHIFT)
    X = tiny_path(pos)
    eng = mop.Engine(sys, precision=prec)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff(X.astype(np.float64), want=("G", "F", "Heta"), hvp_mode=oracle.HVP_ANALYTIC)
    N = X.shape[0]
    tol = 1e-8 if prec == mop.MOP_PREC_FP64 else 1.0
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V * tol
    assert rel(eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1], r["F"][:N - 1]) < TOL_F * tol
    assert rel(eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1], r["Heta"][:N - 1]) < TOL_H * tol
    assert rel(G, r["G"]) < TOL_F * tol
    # the shift changes the energy, not the forces inside rc: V_eff differs from the shifted-force
    # system's by the cutoff terms
    ref = mop.Engine(dataclasses.replace(sys, cutoff_mode=synth.CUTOFF_SHIFTED_FORCE), precision=prec)
    ref.set_path(0, X)
    assert ref.veff_and_grad(0)[0][0] != v[0]


def test_sort_with_equal_and_zero_z_matches_oracle():
    """The spatial sort ranks atoms inside a column by (z of bead 1, atom index).  Four atoms at
    z = 0 exactly and two with equal z (all 13 atoms share one column here) must still get
    distinct slots: any slot collision loses an atom and breaks parity."""
    sys, pos = tiny_system()
    X = tiny_path(pos)
    for a in (6, 7, 8, 9):
        X[0, a, 2] = np.float32(0.0)
    X[0, 11, 2] = X[0, 10, 2]
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff(X.astype(np.float64), want=("G", "F", "Heta"), hvp_mode=oracle.HVP_ANALYTIC)
    N = X.shape[0]
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1], r["F"][:N - 1]) < TOL_F
    assert rel(eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1], r["Heta"][:N - 1]) < TOL_H
    assert rel(G, r["G"]) < TOL_F


def test_tiny_ragged_system_with_spme_matches_oracle():
    sys, pos = tiny_system()
    sys = synth.with_pme(sys)
    X = tiny_path(pos)
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    N = X.shape[0]
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1]
    H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(F, r["F"][:N - 1]) < TOL_F
    assert rel(H, r["Heta"][:N - 1]) < TOL_H
    assert rel(G, r["G"]) < TOL_F


def test_sixty_four_paths_in_one_call():
    w = workload(2, n_beads=3)
    X = w.paths[0]
    rng = np.random.default_rng(3)
    eng = mop.Engine(w.system)
    paths = []
    for p in range(64):
        n = 2 + p % 3                                 # 2..4 beads
        Xp = (X[:1] + rng.normal(0.0, 0.01, (n,) + X.shape[1:])).astype(np.float32)
        eng.set_path(p, Xp)
        paths.append(Xp)
    v_all, G_all = eng.veff_and_grad(-1)
    for p in (0, 1, 31, 62, 63):
        off = sum(q.shape[0] for q in paths[:p])
        v1, G1 = eng.veff_and_grad(p)
        n = paths[p].shape[0]
        assert v1[0] == v_all[p]
        assert np.array_equal(G1, G_all[off:off + n])
    with pytest.raises(mop.MopError) as ei:
        eng.set_path(64, X)
    assert ei.value.status == mop.MOP_ERR_ARG


@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_non_cubic_box_matches_oracle(prec):
    # three different box edges (minimum image, cluster columns and bins per dimension)
    sys, pos = tiny_system(seed=8, box=(2.3, 2.6, 2.9))
    X = tiny_path(pos, seed=4)
    eng = mop.Engine(sys, precision=prec)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff(X.astype(np.float64), want=("G", "F"), hvp_mode=oracle.HVP_ANALYTIC)
    tol = 1e-8 if prec == mop.MOP_PREC_FP64 else 1.0
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V * tol
    assert rel(G, r["G"]) < TOL_F * tol


def test_non_cubic_spme_grid_matches_oracle():
    # K1 != K2 != K3: the grid index order of spreading, the FFT layout, the kernel and gathering
    sys, pos = tiny_system(seed=8, box=(2.3, 2.6, 2.9))
    sys = dataclasses.replace(synth.with_pme(sys), pme_grid=(20, 24, 27))
    X = tiny_path(pos, seed=4)
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    N = X.shape[0]
    H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(G, r["G"]) < TOL_F
    assert rel(H, r["Heta"][:N - 1]) < TOL_H


@pytest.mark.parametrize("N", [1, 2])
@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_one_and_two_bead_paths_match_oracle(N, prec):
    """The shortest paths: one bead (no spring, so V_eff = U(R^1) and the gradient is -F^1) and two
    beads (one spring, one H eta row).  In mixed precision each fills one bead group with 63 or 62
    idle lanes, and the coordinate and list kernels see a single force row."""
    w = workload(2, relaxed=True, n_beads=N)
    X = w.paths[0]
    eng = mop.Engine(w.system, precision=prec)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:1]
    eng.close()
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F"), hvp_mode=oracle.HVP_ANALYTIC)
    # FP64: sums over thousands of pair terms with cancellation round at ~1e-13 of the result
    tol = 1e-6 if prec == mop.MOP_PREC_FP64 else 1.0
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V * tol
    assert rel(G, r["G"]) < TOL_F * tol
    assert rel(F, r["F"][:1]) < TOL_F * tol
    if N == 1:
        assert rel(G, -r["F"][:1]) < TOL_F * tol   # V_eff = U(R^1): the gradient is minus the force
