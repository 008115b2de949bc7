"""Ewald electrostatics (MOP_ELEC_PME) through the C ABI against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import mop, synth
from tests.conftest import workload
from tests.test_gpu_parity import TOL_F, TOL_H, TOL_V, rel

pytestmark = pytest.mark.gpu


def fields(eng, n_beads):
    return dict(F=eng.get_field(0, mop.MOP_FIELD_FORCE)[:n_beads - 1], eta=eng.get_field(0, mop.MOP_FIELD_ETA)[:n_beads - 1],
                Heta=eng.get_field(0, mop.MOP_FIELD_HETA)[:n_beads - 1])


@pytest.mark.parametrize("hvp", [mop.MOP_HVP_ADJOINT, mop.MOP_HVP_FD])
def test_ewald_real_space_matches_oracle(hvp):
    # real space (erfc, cutoff modifier), exclusion corrections and self term; no reciprocal part
    w = workload(2, n_beads=6)
    sys = dataclasses.replace(synth.with_pme(w.system), pme_grid=(0, 0, 0))
    X = w.paths[0]
    eng = mop.Engine(sys, hvp_mode=hvp, fd_h=1e-4)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    g = fields(eng, X.shape[0])
    o = oracle.Oracle(sys)
    r = o.veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"),
               hvp_mode=oracle.HVP_ANALYTIC if hvp == mop.MOP_HVP_ADJOINT else oracle.HVP_FD_EQ5, fd_h=1e-4)
    N = X.shape[0]
    errs = dict(F=rel(g["F"], r["F"][:N - 1]), eta=rel(g["eta"], r["eta"][:N - 1]),
                Heta=rel(g["Heta"], r["Heta"][:N - 1]), G=rel(G, r["G"]), V=abs(v[0] - r["veff"]) / abs(r["veff"]))
    print("ewald real space", hvp, errs)
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["V"] < TOL_V
    if hvp == mop.MOP_HVP_ADJOINT:
        assert errs["Heta"] < TOL_H and errs["G"] < TOL_F
    else:
        # an FP32 central difference at h = 1e-4 nm carries ~1e-4 of its own error (as with the
        # reaction field): the FD path is compared with the oracle's FD of Eq. 5 at that level
        assert errs["Heta"] < 1e-3 and errs["G"] < 1e-3


def pme_errors(eng, path_id, X, v, G, r):
    N = X.shape[0]
    F = eng.get_field(path_id, mop.MOP_FIELD_FORCE)[:N - 1]
    eta = eng.get_field(path_id, mop.MOP_FIELD_ETA)[:N - 1]
    He = eng.get_field(path_id, mop.MOP_FIELD_HETA)[:N - 1]
    return dict(F=rel(F, r["F"][:N - 1]), eta=rel(eta, r["eta"][:N - 1]), Heta=rel(He, r["Heta"][:N - 1]),
                G=rel(G, r["G"]), V=abs(v - r["veff"]) / abs(r["veff"]))


def assert_within_bars(errs):
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["G"] < TOL_F, errs
    assert errs["Heta"] < TOL_H and errs["V"] < TOL_V, errs


def test_spme_matches_oracle():
    # real space, exclusions, self term and the SPME reciprocal part (forces, bead-1 energy and
    # the adjoint H eta through the derivative grid)
    w = workload(2, n_beads=6)
    sys = synth.with_pme(w.system)
    X = w.paths[0]
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    errs = pme_errors(eng, 0, X, v[0], G, r)
    print("spme", sys.pme_grid, errs)
    assert_within_bars(errs)
    # the reciprocal part is not negligible here: without it the oracle's forces differ by far more
    no_recip = oracle.Oracle(dataclasses.replace(sys, pme_grid=(0, 0, 0))).veff(
        X.astype(np.float64), want=("F",), hvp_mode=oracle.HVP_ANALYTIC)
    assert rel(no_recip["F"][:X.shape[0] - 1], r["F"][:X.shape[0] - 1]) > 100 * TOL_F


@pytest.mark.parametrize("order", [6, 7])
def test_spme_higher_orders_match_oracle(order):
    w = workload(2, n_beads=3)
    base = synth.with_pme(w.system, order=order)
    grid = tuple(k + 1 if order % 2 and k % 2 == 0 else k for k in base.pme_grid)   # odd orders: odd grids
    sys = dataclasses.replace(base, pme_grid=grid)
    X = w.paths[0]
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    errs = pme_errors(eng, 0, X, v[0], G, r)
    print("spme order", order, grid, errs)
    assert_within_bars(errs)


def test_spme_uneven_paths_in_one_launch():
    # two paths of different lengths evaluated together (one FFT batch per path)
    w = workload(2, n_beads=6)
    sys = synth.with_pme(w.system)
    paths = [w.paths[0], np.ascontiguousarray(w.paths[0][::-1][:4])]
    eng = mop.Engine(sys)
    for p, X in enumerate(paths):
        eng.set_path(p, X)
    v, G = eng.veff_and_grad(-1)
    o = oracle.Oracle(sys)
    off = 0
    for p, X in enumerate(paths):
        r = o.veff_pme(X.astype(np.float64))
        errs = pme_errors(eng, p, X, v[p], G[off:off + X.shape[0]], r)
        off += X.shape[0]
        print("spme batch", p, errs)
        assert_within_bars(errs)


def test_spme_graph_step_matches_eager_steps():
    # the captured step replays the FFTs and the fixed-point grids bit for bit
    w = workload(2, n_beads=8)
    sys = synth.with_pme(w.system)
    engs = []
    for graph in (False, True):
        eng = mop.Engine(sys)
        eng.set_path(0, w.paths[0])
        eng.set_graph_mode(graph)
        engs.append(eng)
    engs[0].step(4, 1e-5, 2.0, seed=3)
    engs[1].step(4, 1e-5, 2.0, seed=3)
    assert np.array_equal(engs[0].get_path(0), engs[1].get_path(0))
    va, ga = engs[0].veff_and_grad(0)
    vb, gb = engs[1].veff_and_grad(0)
    assert np.array_equal(va, vb) and np.array_equal(ga, gb)
    assert np.isfinite(va).all()


@pytest.mark.parametrize("n_beads", [1, 2])
def test_spme_short_paths_match_oracle(n_beads):
    # N = 1: V_eff = U(R1) with the reciprocal energy, G = -F (no eta, no HVP pass);
    # N = 2: one force bead, one HVP bead
    w = workload(2, n_beads=3)
    sys = synth.with_pme(w.system)
    X = np.ascontiguousarray(w.paths[0][:n_beads])
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(G, r["G"]) < TOL_F
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:max(1, n_beads - 1)]
    assert rel(F, r["F"][:max(1, n_beads - 1)]) < TOL_F
    if n_beads == 1:
        assert rel(G[0], -r["F"][0]) < TOL_F


def test_spme_metadynamics_graph_equals_eager():
    # the production loop on an Ewald system: rounds of MD steps with a Gaussian deposited on a
    # centre-of-mass end-to-end CV after each round, captured (graph) and eager, bit for bit
    w = workload(2, n_beads=6)
    sys = synth.with_pme(w.system)
    X = w.paths[0]
    pos = X[-1].astype(np.float64)
    ga = synth.nearest_group(pos, np.asarray(sys.box), pos[0], 8)
    gb = synth.nearest_group(pos, np.asarray(sys.box), pos[1500], 8)
    runs = []
    for graph in (False, True):
        eng = mop.Engine(sys)
        eng.set_path(0, X)
        eng.add_bias(0, 0.0, 0.0, 0.1, groups=(ga, gb), e2e=True, com=True)
        eng.set_graph_mode(graph)
        eng.metadynamics(3, 2, 1e-6, 5.0, 7, 1.0, 0.1)
        runs.append((eng.get_path(0), eng.gaussians(0), eng.veff_and_grad(0)))
    (x0, g0, (v0, G0)), (x1, g1, (v1, G1)) = runs
    assert len(g0[0]) == 4 and np.isfinite(v0).all()   # the zero-height one plus three deposits
    assert np.array_equal(x0, x1)
    assert np.array_equal(g0[0], g1[0]) and np.array_equal(g0[1], g1[1])
    assert np.array_equal(v0, v1) and np.array_equal(G0, G1)
