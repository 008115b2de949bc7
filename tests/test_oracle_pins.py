"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks a property fixed by the paper (Eqs. 3, 5-7, Sec. 1.1-1.2) or by the
mathematics (closed forms, symmetries, exact derivatives), so that a dropped term, a wrong
sign, a wrong index or a transposed operand in oracle/oracle.cpp fails at least one of them.
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import synth
from tests.conftest import workload

F_COULOMB = 138.935458  # e^2 / (4 pi eps0) in kJ mol^-1 nm e^-2 (physical constant)


def small_system(pos, types, sigma, eps, charge=None, mass=None, box=10.0, rc=1.0, eps_rf=1.0,
                 cutoff_mode=synth.CUTOFF_SHIFTED_FORCE, mol_id=None, mol_local=None,
                 bonds=(), angles=()):
    pos = np.asarray(pos, float)
    Q = len(pos)
    return synth.System(
        box=np.full(3, float(box)), type=np.asarray(types, np.int32),
        lj_sigma=np.asarray(sigma, float), lj_eps=np.asarray(eps, float),
        charge=np.zeros(Q) if charge is None else np.asarray(charge, float),
        mass=np.full(Q, 10.0) if mass is None else np.asarray(mass, float),
        mol_id=np.arange(Q, dtype=np.int32) if mol_id is None else np.asarray(mol_id, np.int32),
        mol_local=np.zeros(Q, np.int32) if mol_local is None else np.asarray(mol_local, np.int32),
        bond_ij=np.asarray([b[:2] for b in bonds], np.int32).reshape(-1, 2),
        bond_r0=np.asarray([b[2] for b in bonds], float), bond_k=np.asarray([b[3] for b in bonds], float),
        angle_ijk=np.asarray([a[:3] for a in angles], np.int32).reshape(-1, 3),
        angle_th0=np.asarray([a[3] for a in angles], float), angle_k=np.asarray([a[4] for a in angles], float),
        rc=rc, eps_rf=eps_rf, cutoff_mode=cutoff_mode)


def pair_U_F(sys, r):
    pos = np.array([[3.0, 3.0, 3.0], [3.0 + r, 3.0, 3.0]])
    o = oracle.Oracle(sys)
    F, U = o.forces(pos)
    return U, F


# --------------------------------------------------------------------------------------------
# random numbers


def test_philox_known_answers():
    path = Path(__file__).parent / "golden" / "philox4x32_10_kat.txt"
    rows = [ln.split() for ln in path.read_text().splitlines() if ln and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        got = oracle.philox4x32_10(v[0:4], v[4:6])
        assert got.tolist() == v[6:10]


def test_gauss3_moments():
    z = np.array([oracle.gauss3(7, 3, b, a) for b in range(4) for a in range(5000)]).ravel()
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    assert abs(np.mean(z ** 4) - 3.0) < 0.15          # Gaussian kurtosis


# --------------------------------------------------------------------------------------------
# single pairs


def test_lj_minimum_and_depth():
    sig, eps = 0.34, 0.996
    s = small_system([[0, 0, 0], [1, 0, 0]], [0, 0], [sig], [eps], rc=3.0,
                     cutoff_mode=synth.CUTOFF_POT_SHIFT)
    rmin = 2.0 ** (1.0 / 6.0) * sig
    U_min, F_min = pair_U_F(s, rmin)
    U_sig, F_sig = pair_U_F(s, sig)
    assert np.abs(F_min).max() < 1e-9                       # minimum of the LJ well
    assert U_min - U_sig == pytest.approx(-eps, rel=1e-12)   # depth eps below the zero crossing
    assert F_sig[0, 0] < 0 < F_sig[1, 0]                     # repulsive inside the minimum


def test_coulomb_difference_and_force():
    q1, q2 = 0.7, -0.4
    s = small_system([[0, 0, 0], [1, 0, 0]], [0, 0], [0.0], [0.0], charge=[q1, q2], rc=2.0,
                     eps_rf=1.0, cutoff_mode=synth.CUTOFF_POT_SHIFT)
    U1, F1 = pair_U_F(s, 0.5)
    U2, _ = pair_U_F(s, 1.25)
    assert U1 - U2 == pytest.approx(F_COULOMB * q1 * q2 * (1 / 0.5 - 1 / 1.25), rel=1e-12)
    # attractive pair: force on atom 0 points to atom 1 with magnitude f|q1 q2|/r^2
    assert F1[0, 0] == pytest.approx(-F_COULOMB * q1 * q2 / 0.25, rel=1e-12)


def test_reaction_field_conducting_boundary_force_vanishes_at_rc():
    s = small_system([[0, 0, 0], [1, 0, 0]], [0, 0], [0.0], [0.0], charge=[1.0, 1.0], rc=1.0,
                     eps_rf=1e15, cutoff_mode=synth.CUTOFF_POT_SHIFT)
    _, F = pair_U_F(s, 1.0 - 1e-9)
    assert abs(F[0, 0]) < 1e-6
    _, F_in = pair_U_F(s, 0.5)
    assert abs(F_in[0, 0]) > 100


@pytest.mark.parametrize("charges", [(0.0, 0.0), (0.5, -0.8)])
def test_shifted_force_vanishes_continuously_at_rc(charges):
    s = small_system([[0, 0, 0], [1, 0, 0]], [0, 0], [0.3], [0.7], charge=list(charges), rc=1.0,
                     eps_rf=78.0)
    for d in (1e-3, 1e-4):
        U, F = pair_U_F(s, 1.0 - d)
        Uo, Fo = pair_U_F(s, 1.0 - 10 * d)
        assert abs(U) < abs(Uo) / 50          # U = O(d^2)
        assert abs(F[0, 0]) < abs(Fo[0, 0]) / 5   # F = O(d)
    U, F = pair_U_F(s, 1.0 + 1e-6)
    assert U == 0.0 and np.all(F == 0.0)


def test_exclusion_rule():
    # same molecule and |local_i - local_j| <= 2 -> excluded; 3 apart -> interacts
    pos = [[2, 2, 2], [2.4, 2, 2], [2, 2.4, 2], [2, 2, 2.4]]
    x = np.array(pos, float)

    def pair_energy(a, b):
        s = small_system([pos[a], pos[b]], [0, 0], [0.3], [1.0])
        return oracle.Oracle(s).forces(np.array([pos[a], pos[b]], float))[1]

    s = small_system(pos, [0] * 4, [0.3], [1.0], mol_id=[0, 0, 0, 0], mol_local=[0, 1, 2, 3])
    U = oracle.Oracle(s).forces(x)[1]
    assert U == pytest.approx(pair_energy(0, 3), rel=1e-14)
    s2 = small_system(pos, [0] * 4, [0.3], [1.0], mol_id=[0, 1, 2, 0], mol_local=[0, 1, 2, 3])
    U2 = oracle.Oracle(s2).forces(x)[1]
    every = sum(pair_energy(a, b) for a in range(4) for b in range(a + 1, 4))
    assert U2 == pytest.approx(every, rel=1e-14)


# --------------------------------------------------------------------------------------------
# bonded terms


def test_bond_hessian_eigenvalues():
    k, r0, d = 345000.0, 0.1, 0.112
    s = small_system([[2, 2, 2], [2 + d, 2, 2]], [0, 0], [0.0], [0.0], mol_id=[0, 0],
                     mol_local=[0, 1], bonds=[(0, 1, r0, k)])
    o = oracle.Oracle(s)
    x = np.array([[2, 2, 2], [2 + d, 2, 2]], float)
    F, U = o.forces(x)
    assert U == pytest.approx(0.5 * k * (d - r0) ** 2, rel=1e-12)
    assert F[0, 0] == pytest.approx(k * (d - r0), rel=1e-12)  # stretched bond pulls atom 0 to +x
    ev = np.sort(np.linalg.eigvalsh(o.hessian(x)))
    expect = np.sort([0, 0, 0, 2 * k, 2 * k * (1 - r0 / d), 2 * k * (1 - r0 / d)])
    np.testing.assert_allclose(ev, expect, atol=1e-6 * k)


def test_angle_energy_and_equilibrium():
    k, th0 = 383.0, np.deg2rad(109.47)
    # vertex at the origin, two arms at 90 degrees
    x = np.array([[3.1, 3.0, 3.0], [3.0, 3.0, 3.0], [3.0, 3.2, 3.0]])
    s = small_system(x, [0] * 3, [0.0], [0.0], mol_id=[0] * 3, mol_local=[0, 1, 2],
                     angles=[(0, 1, 2, th0, k)])
    o = oracle.Oracle(s)
    F, U = o.forces(x)
    assert U == pytest.approx(0.5 * k * (np.pi / 2 - th0) ** 2, rel=1e-12)
    np.testing.assert_allclose(F.sum(0), 0, atol=1e-9)
    torque = np.cross(x - x[1], F).sum(0)
    np.testing.assert_allclose(torque, 0, atol=1e-9)
    # opening the angle toward theta0 lowers U: the force on atom 0 has a -y component
    assert F[0, 1] < 0
    # at theta = theta0 the force vanishes
    x2 = np.array([[3.0 + 0.1, 3.0, 3.0], [3.0, 3.0, 3.0],
                   [3.0 + 0.2 * np.cos(th0), 3.0 + 0.2 * np.sin(th0), 3.0]])
    F2, U2 = o.forces(x2)
    assert U2 < 1e-20 and np.abs(F2).max() < 1e-9


# --------------------------------------------------------------------------------------------
# many-body checks on the seeded workloads


def test_cell_list_matches_brute_force():
    w = workload(2, n_beads=2)
    o = oracle.Oracle(w.system)
    x = w.paths[0][0].astype(float)
    Fc, Uc = o.forces(x, 0)
    Fb, Ub = o.forces(x, 1)
    assert Uc == pytest.approx(Ub, rel=1e-13)
    assert np.abs(Fc - Fb).max() <= 1e-12 * np.abs(Fb).max()


def test_newton_third_law_and_translation():
    w = workload(2, n_beads=2)
    o = oracle.Oracle(w.system)
    x = w.paths[0][0].astype(float)
    F, U = o.forces(x)
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).sum()
    shift = np.array([0.37, -1.91, 2.5])
    F2, U2 = o.forces(x + shift)
    assert U2 == pytest.approx(U, rel=1e-12)
    assert np.abs(F2 - F).max() < 1e-9 * np.abs(F).max()


def lattice_shift(system, every=7):
    """Whole-box shifts for atoms a % every == 0 (the same in every bead): the path and every
    difference R^{n+1} - R^n are unchanged, while their bonds and pairs now reach across the box
    edge in the caller's coordinates."""
    shift = np.zeros((system.n_atoms, 3))
    shift[::every] = np.asarray(system.box) * np.array([1.0, -1.0, 2.0])
    return shift


def test_periodic_images_of_single_atoms_leave_veff_unchanged():
    # U and the spring term depend on positions only through minimum images (bonded terms, pair
    # terms) and through R^{n+1} - R^n, which a per-atom lattice shift keeps
    w = workload(2, n_beads=3)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    r0 = o.veff(X)
    r1 = o.veff(X + lattice_shift(w.system)[None])
    assert r1["veff"] == pytest.approx(r0["veff"], rel=1e-12)
    assert np.abs(r1["G"] - r0["G"]).max() < 1e-9 * np.abs(r0["G"]).max()


def test_force_is_minus_gradient_of_U(rng):
    w = workload(2, n_beads=2)
    o = oracle.Oracle(w.system)
    x = w.paths[0][0].astype(float)
    F, _ = o.forces(x)
    h = 1e-6
    for _ in range(6):
        i, c = rng.integers(x.shape[0]), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd = -(o.forces(xp)[1] - o.forces(xm)[1]) / (2 * h)
        assert fd == pytest.approx(F[i, c], rel=1e-5, abs=1e-4)


def test_perfect_fcc_has_zero_force():
    sys, pos = synth.lj_fcc()
    F, U = oracle.Oracle(sys).forces(pos)
    assert np.abs(F).max() < 1e-10
    assert U < 0


def test_hvp_analytic_matches_complex_step(rng):
    w = workload(2, n_beads=2)
    o = oracle.Oracle(w.system)
    x = w.paths[0][0].astype(float)
    v = rng.normal(size=x.shape)
    Ha = o.hvp(x, v, oracle.HVP_ANALYTIC)
    Hc = o.hvp(x, v, oracle.HVP_COMPLEX)
    assert np.linalg.norm(Ha - Hc) <= 1e-12 * np.linalg.norm(Hc)
    Hf = o.hvp(x, v, oracle.HVP_FD_EQ5, 1e-6)
    assert np.linalg.norm(Hf - Hc) <= 1e-5 * np.linalg.norm(Hc)


def _tiny_water(n=6, L=2.0, seed=3):
    rng = np.random.default_rng(seed)
    b = synth._Builder()
    sites = rng.random((n, 3)) * L
    b.add_waters(sites, rng, 0, 1)
    sys, pos = b.finish(np.full(3, L), [0.3166, 0.0], [0.65, 0.0], rc=0.9, eps_rf=78.0)
    return sys, pos


def test_dense_hessian_symmetric_and_translation_null():
    sys, pos = _tiny_water()
    o = oracle.Oracle(sys)
    H = o.hessian(pos)
    assert np.abs(H - H.T).max() <= 1e-9 * np.abs(H).max()
    for c in range(3):
        t = np.zeros_like(pos)
        t[:, c] = 1.0
        assert np.abs(H @ t.ravel()).max() < 1e-8 * np.abs(H).max()
    # H v from the dense matrix equals the analytic product
    v = np.random.default_rng(1).normal(size=pos.shape)
    np.testing.assert_allclose(H @ v.ravel(), o.hvp(pos, v).ravel(), rtol=1e-10, atol=1e-8)


def test_rotation_identity_isolated_cluster():
    # isolated cluster (no periodic image within rc): H (w x R) = -(w x F)
    sys, pos = _tiny_water(n=5, L=1.2, seed=9)
    sys.box = np.full(3, 20.0)
    pos = pos + 8.0
    o = oracle.Oracle(sys)
    F, _ = o.forces(pos)
    w = np.array([0.3, -0.7, 0.45])
    Hrot = o.hvp(pos, np.cross(w, pos))
    np.testing.assert_allclose(Hrot, -np.cross(w, F), rtol=1e-9, atol=1e-7 * np.abs(F).max())


# --------------------------------------------------------------------------------------------
# effective potential (Eq. 3) and its gradient (Eqs. 5-7)


def _free_particles(Q=5, L=20.0):
    pos = np.array([[2.0 + 3.5 * i, 5.0, 7.0] for i in range(Q)])
    s = small_system(pos, [0] * Q, [0.3], [0.5], mass=np.linspace(2.0, 30.0, Q), box=L, rc=1.0)
    return s, pos


def test_veff_without_potential_is_free_chain():
    s, pos = _free_particles()
    N = 6
    X = pos[None] + np.random.default_rng(2).normal(0, 0.05, (N,) + pos.shape)
    r = oracle.Oracle(s).veff(X)
    K = s.mass * s.nu_path / (2 * s.dt_path)
    dR = np.diff(X, axis=0)
    assert r["U1"] == 0.0
    assert r["veff"] == pytest.approx(0.5 * np.sum(K[None, :, None] * dR ** 2), rel=1e-13)
    G = np.zeros_like(X)            # discrete Laplacian of the open chain
    G[0] = -K[:, None] * dR[0]
    G[1:-1] = K[None, :, None] * (dR[:-1] - dR[1:])
    G[-1] = K[:, None] * dR[-1]
    np.testing.assert_allclose(r["G"], G, rtol=1e-12, atol=1e-9)


def test_veff_single_bead_is_potential():
    w = workload(2, n_beads=2)
    o = oracle.Oracle(w.system)
    X = w.paths[0][:1].astype(float)
    r = o.veff(X)
    F, U = o.forces(X[0])
    assert r["veff"] == pytest.approx(U, rel=1e-14)
    np.testing.assert_allclose(r["G"][0], -F, rtol=1e-13, atol=1e-9)


def test_gradient_matches_complex_step_directional_derivative(rng):
    w = workload(2, n_beads=4)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    G = o.veff(X)["G"]
    for _ in range(2):
        D = rng.normal(size=X.shape)
        dd = o.veff_complex_dir(X, D)
        assert dd == pytest.approx(np.sum(G * D), rel=1e-9)


def test_gradient_matches_central_differences_of_veff(rng):
    w = workload(2, n_beads=3)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    G = o.veff(X)["G"]
    h = 1e-7
    for _ in range(4):
        n, i, c = rng.integers(3), rng.integers(X.shape[1]), rng.integers(3)
        Xp, Xm = X.copy(), X.copy()
        Xp[n, i, c] += h
        Xm[n, i, c] -= h
        fd = (o.veff(Xp, want=())["veff"] - o.veff(Xm, want=())["veff"]) / (2 * h)
        assert fd == pytest.approx(G[n, i, c], rel=2e-4, abs=1e-2 * np.abs(G[n]).mean())


def _separated_waters(n=4, spacing=3.0, seed=4):
    """Waters too far apart to interact: U is bonds + angles only, a smooth function."""
    rng = np.random.default_rng(seed)
    b = synth._Builder()
    sites = np.array([[1.0 + spacing * k, 2.0, 2.0] for k in range(n)])
    b.add_waters(sites, rng, 0, 1)
    L = spacing * n + 2.0
    sys, pos = b.finish(np.full(3, L), [0.3166, 0.0], [0.65, 0.0], rc=0.9, eps_rf=78.0)
    return sys, pos


def test_paper_effective_forces_eq5_to_7_second_order_on_smooth_U():
    sys, pos = _separated_waters()
    X = synth.make_path(pos, 5, 31, std=0.01).astype(float)
    o = oracle.Oracle(sys)
    exact = o.veff(X)["G"]
    errs = []
    for h in (2e-4, 1e-4):
        G = o.veff(X, hvp_mode=oracle.HVP_FD_EQ5, fd_h=h)["G"]
        errs.append(np.linalg.norm(G - exact) / np.linalg.norm(exact))
    assert errs[1] < 1e-7
    assert 3.0 < errs[0] / errs[1] < 5.0     # central difference: error ~ h^2


def test_paper_effective_forces_eq5_to_7_converge_to_exact_gradient():
    # with pair terms the Hessian jumps at rc (the shifted-force potential is C1 there), so
    # the FD error falls only linearly in h; it still converges to the exact gradient
    w = workload(2, n_beads=4)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    exact = o.veff(X)["G"]
    errs = []
    for h in (1e-4, 1e-5):
        G = o.veff(X, hvp_mode=oracle.HVP_FD_EQ5, fd_h=h)["G"]
        errs.append(np.linalg.norm(G - exact) / np.linalg.norm(exact))
    assert errs[1] < 5e-6
    assert errs[1] < errs[0] / 2.5


def test_veff_terms_are_eq3():
    w = workload(2, n_beads=3)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    r = o.veff(X, want=("G", "F", "eta"))
    F0, U0 = o.forces(X[0])
    assert r["U1"] == pytest.approx(U0, rel=1e-14)
    m = w.system.mass
    c = w.system.dt_path / (m * w.system.nu_path)
    # eta^n = R^{n+1} - R^n - L^n with L^n proportional to F^n
    np.testing.assert_allclose(r["eta"][0], X[1] - X[0] - c[:, None] * F0, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------------------------
# bias (Sec. 1.2, Eq. 8) and dynamics (Eq. 4)


def test_bias_gaussian_and_cv_gradient(rng):
    w = workload(4, n_beads=3)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    ga, gb = w.cv_groups
    s, ds = o.cv_distance(X[-1], ga, gb)
    V, G, S = o.bias(X, ga, gb, [s], [1.0], [0.05])
    assert S == pytest.approx(s) and V == pytest.approx(1.0)   # at the centre: height
    assert np.abs(G).max() < 1e-12                             # and zero slope
    V2, G2, _ = o.bias(X, ga, gb, [s - 0.05], [1.0], [0.05])
    assert V2 == pytest.approx(np.exp(-0.5), rel=1e-12)        # one width away
    h = 1e-6
    for k in range(3):
        a = ga[k]
        for c in range(3):
            xp, xm = X[-1].copy(), X[-1].copy()
            xp[a, c] += h
            xm[a, c] -= h
            fd = (o.cv_distance(xp, ga, gb)[0] - o.cv_distance(xm, ga, gb)[0]) / (2 * h)
            assert fd == pytest.approx(ds[a, c], rel=1e-6, abs=1e-9)
    # chain rule: G = dV/ds * ds/dR at the last bead only
    dVds = -np.exp(-0.5) * 1.0 / 0.05
    np.testing.assert_allclose(G2[-1], dVds * ds, rtol=1e-10, atol=1e-12)
    assert np.abs(G2[:-1]).max() == 0.0
    # end-to-end CV of Eq. 8 subtracts s(R^1)
    _, _, S_e2e = o.bias(X, ga, gb, [0.0], [1.0], [0.05], e2e=True)
    assert S_e2e == pytest.approx(s - o.cv_distance(X[0], ga, gb)[0], rel=1e-12)


def test_nve_energy_error_scales_as_dt_squared():
    # velocity Verlet on the path Hamiltonian V_eff + sum m v^2 / 2 (Eq. 4, paper Sec. 2.3 test)
    sys, pos = synth.lj_fcc()
    N = 4
    X0 = synth.make_path(pos, N, 77, std=0.005).astype(float)
    o = oracle.Oracle(sys)
    m = sys.mass[None, :, None]
    drift = []
    T = 0.02
    for dt in (2e-4, 1e-4):
        X = X0.copy()
        V = np.random.default_rng(5).normal(0, 1, X.shape) * np.sqrt(0.0083144626 * 30 / m)
        G = o.veff(X)["G"]
        E0 = o.veff(X, want=())["veff"] + 0.5 * np.sum(m * V ** 2)
        err = 0.0
        for k in range(int(round(T / dt))):
            Ve = o.step(X, V, G, dt, 0.0, 300.0, 1, k, round_f32=False)
            err = max(err, abs(Ve + 0.5 * np.sum(m * V ** 2) - E0))
        drift.append(err)
    assert 3.0 < drift[0] / drift[1] < 5.0


def test_com_cv_reduces_to_centroid_and_matches_two_atom_closed_form():
    # with unit weights the CV is the geometric-centroid distance of the existing pin
    w = workload(4, n_beads=2)
    o = oracle.Oracle(w.system)
    x = w.paths[0][-1].astype(float)
    ga, gb = w.cv_groups
    s0, d0 = o.cv_distance(x, ga, gb)
    s1, d1 = o.cv_com(x, ga, gb, com=False)
    assert s1 == pytest.approx(s0, rel=1e-14)
    np.testing.assert_allclose(d1, d0, rtol=1e-12, atol=1e-15)
    # mass-weighted centres of two two-atom groups, written out by hand
    pos = np.array([[1.0, 2.0, 3.0], [1.4, 2.0, 3.3], [4.0, 4.5, 2.0], [4.2, 4.1, 2.6]])
    m = np.array([1.0, 3.0, 2.0, 6.0])
    sys = small_system(pos, [0, 0, 0, 0], [0.3], [0.0], mass=m, box=20.0)
    o2 = oracle.Oracle(sys)
    ca = (1.0 * pos[0] + 3.0 * pos[1]) / 4.0
    cb = (2.0 * pos[2] + 6.0 * pos[3]) / 8.0
    s, ds = o2.cv_com(pos, [0, 1], [2, 3], com=True)
    assert s == pytest.approx(np.linalg.norm(ca - cb), rel=1e-14)
    u = (ca - cb) / np.linalg.norm(ca - cb)
    np.testing.assert_allclose(ds[1], 3.0 / 4.0 * u, rtol=1e-12)
    np.testing.assert_allclose(ds[3], -6.0 / 8.0 * u, rtol=1e-12)
    # and its derivative by central differences
    h = 1e-6
    for a in range(4):
        for c in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[a, c] += h
            xm[a, c] -= h
            fd = (o2.cv_com(xp, [0, 1], [2, 3], True)[0] - o2.cv_com(xm, [0, 1], [2, 3], True)[0]) / (2 * h)
            assert fd == pytest.approx(ds[a, c], rel=1e-6, abs=1e-9)


def _metad_setup():
    sys, pos = synth.lj_fcc()
    X0 = synth.make_path(pos, 3, 91, std=0.005).astype(np.float64)
    ga, gb = np.arange(0, 4), np.arange(100, 104)
    return sys, X0, ga, gb


def test_metad_with_zero_height_is_plain_dynamics_and_deposits_track_the_cv():
    sys, X0, ga, gb = _metad_setup()
    o = oracle.Oracle(sys)
    dt, gamma, T = 2e-4, 5.0, 300.0
    X, V = X0.copy(), np.zeros_like(X0)
    _, (c, h, w) = o.metad(X, V, dt, gamma, T, 7, 0, 2, 3, ga, gb, 0.0, 0.1, com=True)
    # the same six steps without any bias, and the CV after each block of three
    Y, U = X0.copy(), np.zeros_like(X0)
    G = o.veff(Y.astype(np.float32).astype(np.float64))["G"]
    centres = []
    for k in range(6):
        o.step(Y, U, G, dt, gamma, T, 7, k)
        if k % 3 == 2:
            centres.append(o.cv_com(Y[-1].astype(np.float32).astype(np.float64), ga, gb, True)[0])
    assert np.array_equal(X, Y) and np.array_equal(V, U)
    np.testing.assert_allclose(c, centres, rtol=1e-14)
    assert np.all(h == 0.0) and np.all(w == 0.1)


def test_metad_energy_with_a_static_bias_is_conserved_to_second_order():
    # velocity Verlet on V_eff + V_bias + kinetic energy: a bias force inconsistent with the bias
    # energy would show up as a first-order drift
    sys, X0, ga, gb = _metad_setup()
    o = oracle.Oracle(sys)
    m = sys.mass[None, :, None]
    s0 = o.cv_com(X0[-1], ga, gb, True)[0]
    g = ([s0 + 0.02], [500.0], [0.05])          # a steep Gaussian just past the start
    drift = []
    for dt in (2e-4, 1e-4):
        X = X0.copy()
        V = np.random.default_rng(3).normal(0, 1, X.shape) * np.sqrt(0.0083144626 * 30 / m)
        Vb0, _, _ = o.bias_com(X, ga, gb, *g, com=True)
        E0 = o.veff(X, want=())["veff"] + Vb0 + 0.5 * np.sum(m * V ** 2)
        n = int(round(0.01 / dt))
        # one round of n steps; its deposit has zero height, so it does not change the energy
        Vt, _ = o.metad(X, V, dt, 0.0, 300.0, 1, 0, 1, n, ga, gb, 0.0, 0.05, com=True, gaussians=g,
                        round_f32=False)
        drift.append(abs(Vt + 0.5 * np.sum(m * V ** 2) - E0))
    assert drift[1] > 0 and 3.0 < drift[0] / drift[1] < 5.0


def test_multi_cv_bias_reduces_factorises_and_is_a_gradient():
    w = workload(4, n_beads=3)
    o = oracle.Oracle(w.system)
    X = w.paths[0].astype(float)
    ga, gb = w.cv_groups
    gc_, gd = np.arange(10, 14), np.arange(300, 306)
    # one CV: the single-CV bias
    V1, G1, S1 = o.bias_multi(X, [(ga, gb, True, True)], [[0.3], [0.5]], [[0.05], [0.1]], [2.0, 1.5])
    V0, G0, s0 = o.bias_com(X, ga, gb, [0.3, 0.5], [2.0, 1.5], [0.05, 0.1], e2e=True, com=True)
    assert V1 == pytest.approx(V0, rel=1e-14) and S1[0] == pytest.approx(s0, rel=1e-14)
    np.testing.assert_allclose(G1, G0, rtol=1e-12, atol=1e-15)
    # two CVs, one Gaussian of unit height: the product of the one-dimensional factors
    cvs = [(ga, gb, False, False), (gc_, gd, False, True)]
    _, _, S = o.bias_multi(X, cvs, [[0.0, 0.0]], [[1.0, 1.0]], [0.0])
    c, wd = np.array([S[0] - 0.04, S[1] + 0.1]), np.array([0.05, 0.2])
    V2, G2, _ = o.bias_multi(X, cvs, [c], [wd], [1.0])
    assert V2 == pytest.approx(np.exp(-0.5 * (0.04 / 0.05) ** 2) * np.exp(-0.5 * (0.1 / 0.2) ** 2), rel=1e-12)
    # the gradient by central differences of V at a few coordinates of the last bead
    h = 1e-6
    for a in (ga[0], gb[1], gc_[2], gd[3]):
        for k in range(3):
            xp, xm = X.copy(), X.copy()
            xp[-1, a, k] += h
            xm[-1, a, k] -= h
            fd = (o.bias_multi(xp, cvs, [c], [wd], [1.0])[0] - o.bias_multi(xm, cvs, [c], [wd], [1.0])[0]) / (2 * h)
            assert fd == pytest.approx(G2[-1, a, k], rel=1e-5, abs=1e-9)


def test_multi_cv_metad_with_one_cv_is_the_single_cv_loop():
    sys, X0, ga, gb = _metad_setup()
    o = oracle.Oracle(sys)
    X1, V1 = X0.copy(), np.zeros_like(X0)
    _, (c1, h1, w1) = o.metad(X1, V1, 2e-4, 5.0, 300.0, 7, 0, 2, 3, ga, gb, 30.0, 0.05, com=True)
    X2, V2 = X0.copy(), np.zeros_like(X0)
    _, (c2, w2, h2) = o.metad_multi(X2, V2, 2e-4, 5.0, 300.0, 7, 0, 2, 3, [(ga, gb, False, True)], 30.0, [0.05])
    assert np.array_equal(X1, X2) and np.array_equal(V1, V2)
    np.testing.assert_array_equal(c1, c2[:, 0])
    assert np.array_equal(h1, h2) and np.array_equal(w1, w2[:, 0])
