"""Pins of the oracle's Ewald electrostatics (ELEC_PME) against facts outside the oracle: the
Madelung constant of rock salt, the independence of the Ewald sum from its splitting parameter,
the direct reciprocal-space sum, and exact derivatives.  Test infrastructure, CPU only."""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle import pme
from paper_2501_11962_b300 import synth
from tests.test_oracle_pins import small_system

MADELUNG_NACL = 1.747564594633182   # rock-salt Madelung constant (nearest-neighbour distance)


def ewald_total(o, x, mmax):
    """Full Ewald Coulomb energy: real space + exclusions + self (C++ oracle, LJ off) + direct
    reciprocal sum."""
    F, U = o.forces(x)
    Er, Fr = pme.ewald_recip(x, np.asarray(o.system.charge, float), o.system.box, o.system.ew_beta, mmax)
    return U + Er, F + Fr


def test_rock_salt_madelung_constant():
    a = 0.5640                                  # cubic cell edge; nearest neighbours at a / 2
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    cells = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)])
    na = (cells[:, None, :] + base[None, :, :]).reshape(-1, 3)
    cl = na + np.array([0.5, 0.0, 0.0])
    pos = np.vstack([na, cl]) * a
    q = np.concatenate([np.ones(len(na)), -np.ones(len(cl))])
    sys = small_system(pos, [0] * len(pos), [0.3], [0.0], charge=q, box=2 * a, rc=0.55,
                       cutoff_mode=synth.CUTOFF_POT_SHIFT)
    sys = dataclasses.replace(sys, elec=synth.ELEC_PME, ew_beta=11.0)
    o = oracle.Oracle(sys)
    E, F = ewald_total(o, pos, (16, 16, 16))
    n_pairs = len(na)
    assert E / n_pairs == pytest.approx(-MADELUNG_NACL * pme.F_COULOMB / (a / 2), rel=1e-9)
    assert np.abs(F).max() < 1e-6 * pme.F_COULOMB                  # every ion at a centre of symmetry
    # SPME on a fine grid reproduces the reciprocal part
    sys2 = dataclasses.replace(sys, pme_grid=(48, 48, 48), pme_order=6)
    o2 = oracle.Oracle(sys2)
    Er_spme = o2.recip(pos)[0]
    Er = pme.ewald_recip(pos, q, sys.box, sys.ew_beta, (16, 16, 16))[0]
    assert Er_spme == pytest.approx(Er, rel=1e-6)


def _small_water(n=216, rc=0.9):
    sys, pos = synth.water_box(n, rc, 11)
    return sys, pos.astype(np.float64)


def test_ewald_sum_does_not_depend_on_the_splitting():
    # real space, intramolecular exclusion corrections and self term against the reciprocal sum:
    # their total is the periodic Coulomb energy whatever beta (an error in any part shows up)
    sys, pos = _small_water()
    sys = dataclasses.replace(sys, lj_eps=np.zeros_like(sys.lj_eps), cutoff_mode=synth.CUTOFF_POT_SHIFT,
                              bond_k=np.zeros_like(sys.bond_k), angle_k=np.zeros_like(sys.angle_k))
    totals, forces = [], []
    for beta, mmax in ((5.0, 14), (6.5, 18)):
        o = oracle.Oracle(dataclasses.replace(sys, elec=synth.ELEC_PME, ew_beta=beta))
        E, F = ewald_total(o, pos, (mmax, mmax, mmax))
        totals.append(E)
        forces.append(F)
    assert totals[1] == pytest.approx(totals[0], rel=2e-8)
    assert np.abs(forces[1] - forces[0]).max() < 1e-5 * np.abs(forces[0]).max()


def test_spme_converges_to_the_ewald_sum():
    sys, pos = _small_water()
    q = np.asarray(sys.charge, float)
    beta = 3.2
    Er, Fr = pme.ewald_recip(pos, q, sys.box, beta, (14, 14, 14))
    errs = []
    for K, p in ((16, 4), (24, 4), (32, 6)):
        E, F = pme.spme(pos, q, sys.box, (K, K, K), p, beta)
        errs.append(np.linalg.norm(F - Fr) / np.linalg.norm(Fr))
        assert E == pytest.approx(Er, rel=10 * errs[-1] + 1e-7)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-5


def test_spme_forces_and_hessian_vector_product_are_derivatives():
    rng = np.random.default_rng(2)
    sys, pos = _small_water(64, rc=0.55)
    q = np.asarray(sys.charge, float)
    K, p, beta = (20, 20, 20), 4, 4.0
    v = rng.normal(size=pos.shape)
    E, F, H = pme.spme(pos, q, sys.box, K, p, beta, v=v)
    h = 1e-6
    for i in (0, 7, 100):
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g = (pme.spme(xp, q, sys.box, K, p, beta)[0] - pme.spme(xm, q, sys.box, K, p, beta)[0]) / (2 * h)
            assert -g == pytest.approx(F[i, d], rel=1e-6, abs=1e-6)
    h = 1e-5
    Fp = pme.spme(pos + h * v, q, sys.box, K, p, beta)[1]
    Fm = pme.spme(pos - h * v, q, sys.box, K, p, beta)[1]
    assert np.linalg.norm(H + (Fp - Fm) / (2 * h)) < 1e-7 * np.linalg.norm(H)


def test_ewald_real_space_hessian_three_ways():
    # analytic blocks (phi'', exclusion corrections) against the complex step and central
    # differences of the forces
    rng = np.random.default_rng(5)
    sys, pos = _small_water(64, rc=0.55)
    o = oracle.Oracle(synth.with_pme(sys))
    v = rng.normal(size=pos.shape)
    Ha = o.hvp(pos, v, oracle.HVP_ANALYTIC)
    Hc = o.hvp(pos, v, oracle.HVP_COMPLEX)
    Hf = o.hvp(pos, v, oracle.HVP_FD_EQ5, 1e-6)
    assert np.linalg.norm(Ha - Hc) < 1e-9 * np.linalg.norm(Ha)
    assert np.linalg.norm(Ha - Hf) < 1e-5 * np.linalg.norm(Ha)


def test_pme_path_gradient_matches_central_differences():
    rng = np.random.default_rng(8)
    sys, pos = _small_water(27, rc=0.45)
    sys = synth.with_pme(sys, spacing=0.1)
    X = synth.make_path(pos, 3, 41, std=0.004).astype(np.float64)
    o = oracle.Oracle(sys)
    r = o.veff_pme(X)
    h = 1e-6
    for n, i, d in ((0, 3, 0), (1, 10, 2), (2, 40, 1), (1, 0, 1)):
        Xp, Xm = X.copy(), X.copy()
        Xp[n, i, d] += h
        Xm[n, i, d] -= h
        g = (o.veff_pme(Xp)["veff"] - o.veff_pme(Xm)["veff"]) / (2 * h)
        assert g == pytest.approx(r["G"][n, i, d], rel=2e-5, abs=1e-3)
