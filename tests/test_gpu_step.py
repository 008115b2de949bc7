"""mop_step (path dynamics of Eq. 4) against the oracle's integrator.

Both sides draw the Langevin noise from their own Philox-4x32-10 implementation with the same
(seed, step, bead, atom) counters, so BAOAB trajectories agree to rounding; velocity Verlet
conserves V_eff + kinetic energy (the paper's NVE check, Sec. 2.3).
"""
import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu


def run_both(gamma, n_steps=5, dt=2e-4, seed=11):
    w = workload(1, n_beads=4)
    X0 = w.paths[0]
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    eng.set_path(0, X0)
    eng.step(n_steps, dt, gamma, seed)
    Xg = eng.get_path(0).astype(np.float64)
    keg = eng.kinetic_energy(0)
    o = oracle.Oracle(w.system)
    X = X0.astype(np.float64).copy()
    V = np.zeros_like(X)
    G = o.veff(X)["G"]
    for k in range(n_steps):
        o.step(X, V, G, dt, gamma, w.system.temperature, seed, k, round_f32=False)
    ke = 0.5 * np.sum(w.system.mass[None, :, None] * V ** 2)
    return Xg, X, keg, ke


def test_velocity_verlet_matches_oracle():
    Xg, X, keg, ke = run_both(gamma=0.0)
    disp = np.abs(X - workload(1, n_beads=4).paths[0]).max()
    assert disp > 1e-6                                  # the atoms did move
    assert np.abs(Xg - X).max() < 1e-6                  # float32 readback of FP64 positions
    assert keg == pytest.approx(ke, rel=1e-9)


def test_baoab_matches_oracle_noise():
    Xg, X, keg, ke = run_both(gamma=5.0)
    assert np.abs(Xg - X).max() < 1e-6
    assert keg == pytest.approx(ke, rel=1e-8)


def test_nve_energy_conserved():
    w = workload(1, n_beads=4)
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    eng.set_path(0, w.paths[0])
    v0, _ = eng.veff_and_grad(0)
    E0 = v0[0]
    drift = []
    for dt in (2e-4, 1e-4):
        eng.set_path(0, w.paths[0])
        errs = []
        for k in range(int(round(0.004 / dt))):
            eng.step(1, dt, 0.0, 1)
            v, _ = eng.veff_and_grad(0)
            errs.append(abs(v[0] + eng.kinetic_energy(0) - E0))
        drift.append(max(errs))
    assert drift[1] < drift[0]
    assert 2.5 < drift[0] / drift[1] < 5.5           # second-order integrator


@pytest.mark.parametrize("com,graph", [(False, False), (True, False), (True, True)])
def test_metadynamics_matches_oracle(com, graph):
    # three rounds of two BAOAB steps, a Gaussian deposited on the CV after each round, on top of
    # one Gaussian placed by hand; the oracle runs the same loop (same Philox counters)
    w = workload(1, n_beads=4)
    X0 = w.paths[0]
    ga, gb = np.arange(0, 4), np.arange(100, 104)
    o = oracle.Oracle(w.system)
    s0 = o.cv_com(X0[-1].astype(np.float64), ga, gb, com)[0]
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    eng.set_path(0, X0)
    eng.add_bias(0, s0 + 0.02, 20.0, 0.05, groups=(ga, gb), com=com)
    eng.set_graph_mode(graph)
    eng.metadynamics(3, 2, 2e-4, 5.0, 11, 10.0, 0.05)
    Xg = eng.get_path(0).astype(np.float64)
    c, h, wd = eng.gaussians(0)
    X = X0.astype(np.float64).copy()
    V = np.zeros_like(X)
    _, (co, ho, wo) = o.metad(X, V, 2e-4, 5.0, w.system.temperature, 11, 0, 3, 2, ga, gb, 10.0, 0.05, com=com,
                              gaussians=([s0 + 0.02], [20.0], [0.05]), round_f32=False)
    assert len(c) == 4 and np.abs(X - X0).max() > 1e-6
    assert np.abs(Xg - X).max() < 1e-6                  # float32 readback of FP64 positions
    np.testing.assert_allclose(c[:, 0], co, rtol=1e-10)
    assert np.array_equal(h, ho) and np.array_equal(wd[:, 0], wo)


def test_multi_cv_metadynamics_matches_oracle():
    # two CVs (a centre-of-mass end-to-end distance with its own deposit width, and a plain
    # centroid distance) with multivariate Gaussians, deposited in graph mode
    w = workload(1, n_beads=4)
    X0 = w.paths[0]
    cvs = [(np.arange(0, 4), np.arange(100, 104), True, True), (np.arange(20, 26), np.arange(200, 203), False, False)]
    o = oracle.Oracle(w.system)
    _, _, S0 = o.bias_multi(X0.astype(np.float64), cvs, [[0.0, 0.0]], [[1.0, 1.0]], [0.0])
    g0 = ([[S0[0] + 0.01, S0[1] - 0.02]], [[0.05, 0.08]], [15.0])
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    eng.set_path(0, X0)
    assert eng.add_cv(0, cvs[0][:2], e2e=True, com=True, deposit_width=0.03) == 0
    assert eng.add_cv(0, cvs[1][:2]) == 1
    eng.add_gaussian(0, 15.0, g0[0][0], g0[1][0])
    eng.set_graph_mode(True)
    eng.metadynamics(2, 3, 2e-4, 5.0, 17, 8.0, 0.06)
    Xg = eng.get_path(0).astype(np.float64)
    c, h, wd = eng.gaussians(0)
    X = X0.astype(np.float64).copy()
    V = np.zeros_like(X)
    _, (co, wo, ho) = o.metad_multi(X, V, 2e-4, 5.0, w.system.temperature, 17, 0, 2, 3, cvs, 8.0, [0.03, 0.06],
                                    gaussians=g0, round_f32=False)
    assert c.shape == (3, 2) and np.abs(X - X0).max() > 1e-6
    assert np.abs(Xg - X).max() < 1e-6
    np.testing.assert_allclose(c, co, rtol=1e-10)
    assert np.array_equal(h, ho) and np.array_equal(wd, wo)


def test_baoab_thermostat_holds_the_temperature():
    # NVT check of the path dynamics (the paper's Sec. 2.3 validation): with strong Langevin
    # coupling the kinetic temperature of all beads settles at the bath temperature
    # (equipartition, 3 degrees of freedom per atom and bead)
    w = workload(1, n_beads=4)
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    eng.set_path(0, w.paths[0])
    T, dt, gamma = w.system.temperature, 2e-4, 50.0
    eng.step(200, dt, gamma, 5)                      # about 10 / gamma to equilibrate
    kin = []
    for _ in range(40):
        eng.step(5, dt, gamma, 5)
        kin.append(eng.kinetic_energy(0))
    dof = 3 * w.system.n_atoms * w.paths[0].shape[0]
    T_kin = 2.0 * np.mean(kin) / (dof * 0.0083144626)
    assert abs(T_kin - T) / T < 0.05, T_kin


@pytest.mark.parametrize("gamma", [0.0, 5.0])
def test_deferred_integrator_state_matches_eager(gamma):
    """Mixed precision with float input: mop_set_path leaves the FP64 integrator copy and the zero
    velocities to the first mop_step.  The trajectory must equal, bit for bit, the one from the
    same coordinates given as doubles (whose integrator copy mop_set_path forms at once), and
    again after a second mop_set_path on a handle that has already stepped."""
    w = workload(2, n_beads=4)
    X32 = np.ascontiguousarray(w.paths[0], dtype=np.float32)
    X64 = X32.astype(np.float64)
    out = []
    for X in (X32, X64):
        eng = mop.Engine(w.system)
        eng.set_path(0, X)
        assert eng.kinetic_energy(0) == 0.0
        eng.step(3, 2e-4, gamma, 7)
        a = eng.get_path(0)
        ke_a = eng.kinetic_energy(0)
        eng.set_path(0, X)                  # back to the start: positions and velocities reset
        assert eng.kinetic_energy(0) == 0.0
        eng.step(3, 2e-4, gamma, 7)
        b = eng.get_path(0)
        out.append((a, ke_a, b))
        eng.close()
    (a32, ke32, b32), (a64, ke64, b64) = out
    assert np.abs(a32 - X32).max() > 0.0    # the atoms moved
    assert np.array_equal(a32, a64) and ke32 == ke64
    assert np.array_equal(b32.view(np.uint32), b64.view(np.uint32))
