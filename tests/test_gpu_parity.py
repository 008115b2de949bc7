"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative 2-norms over all beads and atoms, the required accuracy):
  forces F^n <= 1e-5, H eta <= 1e-4, V_eff <= 1e-6 (mixed precision);
  FP64 mode: 1e-9.
The gradient G, eta and the energy parts are reported and held to the same bars as the
quantity that dominates them (F for eta and G, V_eff for the energies).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu

TOL_F, TOL_H, TOL_V = 1e-5, 1e-4, 1e-6
TOL_F64 = 1e-9


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


U32 = 2.0 ** -24   # FP32 unit roundoff


def row_rel(a, b):
    """Per-row (atom and bead) relative errors |a_i - b_i| / |b_i|, each row's norm floored at 1e-3
    of the RMS row norm so that near-zero rows do not dominate."""
    a = np.asarray(a, np.float64).reshape(-1, 3)
    b = np.asarray(b, np.float64).reshape(-1, 3)
    nb = np.linalg.norm(b, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nb ** 2))
    return np.linalg.norm(a - b, axis=1) / np.maximum(nb, floor)


def assert_rows(a, b, bar, name):
    """A localized error (a missed pair, a wrong exclusion bit) hides in a norm over millions of
    rows; the 99.9th percentile of the per-row error must also stay within ten times the bar."""
    r = row_rel(a, b)
    q = float(np.quantile(r, 0.999))
    print(f"{name}: rows {r.size}, 99.9th percentile {q:.2e}, max {r.max():.2e}")
    assert q < 10 * bar, (name, q)


def gpu_eval(w, path=0, **kw):
    eng = mop.Engine(w.system, **kw)
    eng.set_path(path, w.paths[0])
    v, G = eng.veff_and_grad(path)
    out = dict(veff=v[0], G=G, F=eng.get_field(path, mop.MOP_FIELD_FORCE),
               eta=eng.get_field(path, mop.MOP_FIELD_ETA), Heta=eng.get_field(path, mop.MOP_FIELD_HETA))
    out.update(eng.energies(path))
    out["launches"] = eng.last_launch_count()
    return eng, out


def test_cfg1_fp64_matches_oracle():
    w = workload(1)
    X = w.paths[0]
    eng, g = gpu_eval(w, precision=mop.MOP_PREC_FP64)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"))
    N = X.shape[0]
    errs = dict(F=rel(g["F"][:N - 1], r["F"][:N - 1]), eta=rel(g["eta"][:N - 1], r["eta"][:N - 1]),
                Heta=rel(g["Heta"][:N - 1], r["Heta"][:N - 1]), G=rel(g["G"], r["G"]),
                V=abs(g["veff"] - r["veff"]) / abs(r["veff"]), U1=abs(g["U1"] - r["U1"]) / abs(r["U1"]))
    print("cfg1 fp64 errors", errs)
    for k, e in errs.items():
        assert e < TOL_F64, (k, e)
    assert g["launches"] > 0


@pytest.mark.parametrize("relaxed", [False, True])
def test_cfg2_mixed_matches_oracle(relaxed):
    w = workload(2, relaxed=relaxed)
    X = w.paths[0]
    eng, g = gpu_eval(w)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"))
    N = X.shape[0]
    errs = dict(F=rel(g["F"][:N - 1], r["F"][:N - 1]), eta=rel(g["eta"][:N - 1], r["eta"][:N - 1]),
                Heta=rel(g["Heta"][:N - 1], r["Heta"][:N - 1]), G=rel(g["G"], r["G"]),
                V=abs(g["veff"] - r["veff"]) / abs(r["veff"]), U1=abs(g["U1"] - r["U1"]) / abs(r["U1"]),
                Es=abs(g["Espring"] - r["Espring"]) / abs(r["Espring"]))
    print("cfg2 mixed errors", errs)
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["G"] < TOL_F
    assert errs["Heta"] < TOL_H
    assert errs["V"] < TOL_V and errs["Es"] < TOL_V and errs["U1"] < TOL_V
    assert_rows(g["F"][:N - 1], r["F"][:N - 1], TOL_F, "F")
    assert_rows(g["eta"][:N - 1], r["eta"][:N - 1], TOL_F, "eta")
    assert_rows(g["Heta"][:N - 1], r["Heta"][:N - 1], TOL_H, "Heta")
    assert_rows(g["G"], r["G"], TOL_F, "G")


@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_bonds_across_the_box_edge(prec):
    # every 7th atom moved by whole box vectors in all beads: its bonds and angles cross the box
    # edge in the caller's coordinates, which takes the minimum-image branch of the bonded terms
    from tests.test_oracle_pins import lattice_shift
    w = workload(2, n_beads=6)
    X = (w.paths[0].astype(np.float64) + lattice_shift(w.system)[None]).astype(np.float32)
    eng = mop.Engine(w.system, precision=prec)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)
    H = eng.get_field(0, mop.MOP_FIELD_HETA)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "Heta"))
    N = X.shape[0]
    errs = dict(F=rel(F[:N - 1], r["F"][:N - 1]), Heta=rel(H[:N - 1], r["Heta"][:N - 1]), G=rel(G, r["G"]),
                V=abs(v[0] - r["veff"]) / abs(r["veff"]))
    print("shifted atoms", prec, errs)
    tf, th, tv = (TOL_F, TOL_H, TOL_V) if prec == mop.MOP_PREC_MIXED else (TOL_F64, TOL_F64, TOL_F64)
    assert errs["F"] < tf and errs["G"] < tf and errs["Heta"] < th and errs["V"] < tv, errs


def test_cfg2_small_path_edge_cases():
    """N = 1 (V = U, G = -F) and N = 2 (one spring, no interior bead)."""
    w = workload(2)
    o = oracle.Oracle(w.system)
    eng = mop.Engine(w.system)
    for N in (1, 2):
        X = w.paths[0][:N]
        eng.set_path(0, X)
        v, G = eng.veff_and_grad(0)
        r = o.veff(X.astype(np.float64))
        assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
        assert rel(G, r["G"]) < TOL_F


def test_fd_mode_fp64_matches_oracle_eq5():
    w = workload(1)
    X = w.paths[0]
    eng, g = gpu_eval(w, precision=mop.MOP_PREC_FP64, hvp_mode=mop.MOP_HVP_FD, fd_h=1e-4)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), hvp_mode=oracle.HVP_FD_EQ5, fd_h=1e-4,
                                     want=("G", "Heta"))
    N = X.shape[0]
    assert rel(g["Heta"][:N - 1], r["Heta"][:N - 1]) < 1e-6
    assert rel(g["G"], r["G"]) < 1e-8


@pytest.mark.parametrize("h", [1e-4, 1e-3])
def test_fd_mode_mixed_matches_oracle_eq5(h):
    """The FP32 FD-HVP kernel (the comparison path) against the oracle's own Eq. 5 at the same h
    and the same per-bead eps = h / max_i |eta_i| (reading 4), element by element.  Both sides
    then carry the same truncation error, and what remains is the kernel's FP32 rounding: each
    pair force at R +- eps eta is rounded to about u |f|, and the difference is divided by 2 eps,
    so the scale per bead is u ||F^n|| / (2 eps_n), relative to ||H eta||.  The test allows 30
    times that scale: about ten FP32 operations per pair force, and per-atom sums of |f_ij| that
    exceed |F_i| where the pair forces cancel.  A wrong eps (a factor of 2 changes the truncation
    error fourfold: 2e-2 at h = 1e-3, 3e-4 at h = 1e-4), a sign error in one displaced evaluation
    or a missing bonded FD term exceed it.  G carries H eta / 2, so its bar is the gradient bar
    plus the same allowance scaled by ||H eta|| / (2 ||G||)."""
    w = workload(2)
    X = w.paths[0]
    N = X.shape[0]
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), hvp_mode=oracle.HVP_FD_EQ5, fd_h=h,
                                     want=("G", "F", "eta", "Heta"))
    eng, g = gpu_eval(w, hvp_mode=mop.MOP_HVP_FD, fd_h=h)
    eps = h / np.linalg.norm(r["eta"][:N - 1], axis=2).max(axis=1)
    Fn = np.linalg.norm(r["F"][:N - 1].reshape(N - 1, -1), axis=1)
    bound = U32 * np.sqrt(np.sum((Fn / (2.0 * eps)) ** 2)) / np.linalg.norm(r["Heta"][:N - 1])
    e = rel(g["Heta"][:N - 1], r["Heta"][:N - 1])
    eg = rel(g["G"], r["G"])
    tol = 30.0 * bound
    tol_g = TOL_F + tol * np.linalg.norm(r["Heta"]) / (2.0 * np.linalg.norm(r["G"]))
    print(f"FD h={h:g}: H eta error vs the oracle's Eq. 5 {e:.3e} (FP32 rounding scale {bound:.3e}, "
          f"allowed {tol:.3e}); G {eg:.3e} (allowed {tol_g:.3e})")
    assert e < tol, (e, tol)
    assert eg < tol_g, (eg, tol_g)
    # per row: the FD error is absolute (a rounding of the pair forces divided by 2 eps), so each
    # row is measured in its own rounding scale u max(|F_i|, rms_i |F|) / (2 eps_n); a dropped pair
    # or a wrong sign in one row stands out by orders of magnitude
    Fr = np.linalg.norm(r["F"][:N - 1], axis=2)
    scale = U32 * np.maximum(Fr, np.sqrt(np.mean(Fr ** 2, axis=1))[:, None]) / (2.0 * eps[:, None])
    ratio = np.linalg.norm(g["Heta"][:N - 1] - r["Heta"][:N - 1], axis=2) / scale
    q = float(np.quantile(ratio, 0.999))
    print(f"FD h={h:g}: per-row error in units of the row's rounding scale: 99.9th percentile {q:.1f}, "
          f"max {ratio.max():.1f}")
    assert q < 300.0, q


def test_fd_mode_mixed_accuracy_is_reported():
    w = workload(2)
    X = w.paths[0]
    exact = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "Heta"))
    N = X.shape[0]
    for h in (1e-5, 1e-4, 1e-3):
        eng, g = gpu_eval(w, hvp_mode=mop.MOP_HVP_FD, fd_h=h)
        e = rel(g["Heta"][:N - 1], exact["Heta"][:N - 1])
        print(f"FD h={h:g}: H eta error vs exact {e:.3e}, G error {rel(g['G'], exact['G']):.3e}")
        assert np.isfinite(e) and e < 1.0


def test_deterministic_and_batch_invariant():
    w = workload(4, n_beads=8)
    eng = mop.Engine(w.system)
    for p in range(3):
        eng.set_path(p, w.paths[p])
    v_all, G_all = eng.veff_and_grad(-1)
    v_again, G_again = eng.veff_and_grad(-1)
    assert np.array_equal(v_all, v_again) and np.array_equal(G_all, G_again)
    off = 0
    for p in range(3):
        v1, G1 = eng.veff_and_grad(p)
        n = w.paths[p].shape[0]
        assert v1[0] == v_all[p]
        assert np.array_equal(G1, G_all[off:off + n])
        off += n


def test_nonfinite_input_rejected():
    w = workload(2, n_beads=2)
    eng = mop.Engine(w.system)
    X = w.paths[0].copy()
    X[1, 5, 2] = np.nan
    with pytest.raises(mop.MopError) as ei:
        eng.set_path(0, X)
    assert ei.value.status == mop.MOP_ERR_NONFINITE
    with pytest.raises(mop.MopError) as ei:
        eng.veff_and_grad(3)
    assert ei.value.status == mop.MOP_ERR_STATE


@pytest.mark.slow
def test_cfg3_autograd_matches_oracle():
    import torch
    w = workload(3)
    X = w.paths[0]
    eng = mop.Engine(w.system)
    coords = torch.tensor(X, device="cuda", requires_grad=True)
    V = mop.veff(coords, eng, 0)
    V.backward()
    torch.cuda.synchronize()
    G = coords.grad.double().cpu().numpy()
    r = oracle.Oracle(w.system).veff(X.astype(np.float64))
    assert abs(V.item() - r["veff"]) / abs(r["veff"]) < TOL_V
    # float32 gradient from backward: bounded by its own rounding and the FP64 bar
    assert rel(G, r["G"]) < TOL_F


@pytest.mark.slow
def test_cfg4_uneven_batch_with_bias():
    w = workload(4)
    o = oracle.Oracle(w.system)
    eng = mop.Engine(w.system)
    ga, gb = w.cv_groups
    for p, X in enumerate(w.paths):
        eng.set_path(p, X)
        s0, _ = o.cv_distance(X[-1].astype(np.float64), ga, gb)
        eng.add_bias(p, s0 + 0.02, w.bias["height"], w.bias["width"], groups=(ga, gb))
    v, G = eng.veff_and_grad(-1)
    offs = np.cumsum([0] + [X.shape[0] for X in w.paths])
    for p in (0, 1, 4):
        X = w.paths[p].astype(np.float64)
        r = o.veff(X)
        s0, _ = o.cv_distance(X[-1], ga, gb)
        Vb, Gb, S = o.bias(X, ga, gb, [s0 + 0.02], [w.bias["height"]], [w.bias["width"]])
        ref_v = r["veff"] + Vb
        ref_G = r["G"] + Gb
        assert abs(v[p] - ref_v) / abs(ref_v) < TOL_V
        assert rel(G[offs[p]:offs[p + 1]], ref_G) < TOL_F
        e = eng.energies(p)
        assert e["Ebias"] == pytest.approx(Vb, rel=1e-6, abs=1e-9)
        assert e["cv"] == pytest.approx(S, rel=1e-9)


@pytest.mark.parametrize("prec", [mop.MOP_PREC_MIXED, mop.MOP_PREC_FP64])
def test_multi_cv_bias_matches_oracle(prec):
    # two CVs and three multivariate Gaussians on the water box
    w = workload(2, n_beads=5)
    X = w.paths[0]
    pos = X[-1].astype(np.float64)
    cvs = [(np.arange(0, 6), np.arange(300, 309), True, True), (np.arange(900, 903), np.arange(1500, 1506), False, False)]
    o = oracle.Oracle(w.system)
    _, _, S = o.bias_multi(X.astype(np.float64), cvs, [[0.0, 0.0]], [[1.0, 1.0]], [0.0])
    cen = [[S[0] + 0.02, S[1]], [S[0], S[1] - 0.03], [S[0] - 0.05, S[1] + 0.04]]
    wid = [[0.05, 0.06], [0.04, 0.05], [0.06, 0.07]]
    hei = [30.0, 20.0, 25.0]
    eng = mop.Engine(w.system, precision=prec)
    eng.set_path(0, X)
    for ga, gb, e2e, com in cvs:
        eng.add_cv(0, (ga, gb), e2e=e2e, com=com)
    for c_, w_, h_ in zip(cen, wid, hei):
        eng.add_gaussian(0, h_, c_, w_)
    v, G = eng.veff_and_grad(0)
    r = o.veff(X.astype(np.float64))
    Vb, Gb, Sb = o.bias_multi(X.astype(np.float64), cvs, cen, wid, hei)
    assert Vb > 1.0
    tv, tf = (TOL_V, TOL_F) if prec == mop.MOP_PREC_MIXED else (TOL_F64, TOL_F64)
    assert abs(v[0] - (r["veff"] + Vb)) / abs(r["veff"]) < tv
    assert rel(G, r["G"] + Gb) < tf
    e = eng.energies(0)
    assert e["Ebias"] == pytest.approx(Vb, rel=1e-6) and e["cv"] == pytest.approx(Sb[0], rel=1e-9)
    if prec == mop.MOP_PREC_FP64:
        # the rest of the gradient agrees to rounding, so the bias gradient shows on its own
        idx = np.concatenate([c[0] for c in cvs] + [c[1] for c in cvs])
        np.testing.assert_allclose((G - r["G"])[[0, -1]][:, idx], Gb[[0, -1]][:, idx], rtol=1e-7, atol=1e-8)


@pytest.mark.slow
@pytest.mark.parametrize("relaxed", [False, True])
def test_cfg5_sampled_beads_match_oracle(relaxed):
    w = workload(5, relaxed=relaxed)
    X = w.paths[0]
    N = X.shape[0]
    eng, g = gpu_eval(w)
    o = oracle.Oracle(w.system)
    Xd = X.astype(np.float64)
    beads = list(range(N - 1))
    with ThreadPoolExecutor(max_workers=max(1, oracle.num_threads())) as ex:
        res = list(ex.map(lambda n: o.forces(Xd[n]), beads))
    F = np.stack([r[0] for r in res])
    U1 = res[0][1]
    m = w.system.mass
    K = m * w.system.nu_path / (2 * w.system.dt_path)
    c = w.system.dt_path / (m * w.system.nu_path)
    eta = Xd[1:] - Xd[:-1] - c[None, :, None] * F
    Es = 0.5 * np.sum(K[None, :, None] * eta ** 2)
    errs = dict(F=rel(g["F"][:N - 1], F), eta=rel(g["eta"][:N - 1], eta), U1=abs(g["U1"] - U1) / abs(U1),
                V=abs(g["veff"] - (U1 + Es)) / abs(U1 + Es))
    # H eta on 8 beads: both ends, both halves of a lane's pair (beads 31 and 32 share lane 31),
    # and the interior
    sample = [0, 1, 9, 21, 31, 32, 45, N - 2]
    with ThreadPoolExecutor(max_workers=8) as ex:
        H = list(ex.map(lambda n: o.hvp(Xd[n], eta[n]), sample))
    errs["Heta"] = rel(g["Heta"][sample], np.stack(H))
    # gradient on the sampled beads (G^1 for bead index 0) and on bead N
    Gs, Gg = [], []
    for k, n in enumerate(sample):
        Gs.append(-F[0] - K[:, None] * eta[0] + 0.5 * H[k] if n == 0 else
                  K[:, None] * eta[n - 1] - K[:, None] * eta[n] + 0.5 * H[k])
        Gg.append(g["G"][n])
    Gs.append(K[:, None] * eta[N - 2])
    Gg.append(g["G"][N - 1])
    errs["G"] = rel(np.stack(Gg), np.stack(Gs))
    print("cfg5 errors", errs)
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["G"] < TOL_F
    assert errs["Heta"] < TOL_H
    assert errs["V"] < TOL_V and errs["U1"] < TOL_V
    assert_rows(g["F"][:N - 1], F, TOL_F, "cfg5 F")
    assert_rows(g["eta"][:N - 1], eta, TOL_F, "cfg5 eta")
    assert_rows(g["Heta"][sample], np.stack(H), TOL_H, "cfg5 Heta")
    assert_rows(np.stack(Gg), np.stack(Gs), TOL_F, "cfg5 G")


def test_autograd_gradient_matches_central_differences():
    """The torch.autograd.Function's gradient against a central difference of V_eff itself along
    random directions (FP64 mode and FP64 coordinates, so the difference is not drowned in
    rounding)."""
    import torch
    w = workload(1, n_beads=6)
    X = torch.tensor(w.paths[0], dtype=torch.float64, device="cuda")
    eng = mop.Engine(w.system, precision=mop.MOP_PREC_FP64)
    c = X.clone().requires_grad_(True)
    V = mop.veff(c, eng, 0)
    V.backward()
    G = c.grad.detach()
    rng = np.random.default_rng(17)
    h = 1e-5
    for _ in range(3):
        D = torch.tensor(rng.normal(size=tuple(X.shape)), dtype=torch.float64, device="cuda")
        D /= torch.linalg.norm(D)
        with torch.no_grad():
            vp = mop.veff(X + h * D, eng, 0).item()
            vm = mop.veff(X - h * D, eng, 0).item()
        fd = (vp - vm) / (2.0 * h)
        an = float((G * D).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)


def test_spread_out_beads_skip_empty_halves_and_match_oracle():
    """Beads 4..6 of the path are those of beads 1..3 moved by 0.25 nm along x.  The list, built
    from each atom's union over all beads, then holds many half-clusters that have no pair within
    rc for a given bead pair; the pair kernels skip those by warp vote and clear their bits for
    the j-side flush (the force, adjoint H eta and FD kernels).  Results match the oracle."""
    w = workload(2, n_beads=3)
    X3 = w.paths[0]
    X = np.concatenate([X3, X3 + np.float32(0.25) * np.array([1.0, 0.0, 0.0], np.float32)]).astype(np.float32)
    N = X.shape[0]
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "Heta"), hvp_mode=oracle.HVP_ANALYTIC)
    eng = mop.Engine(w.system)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    assert abs(v[0] - r["veff"]) / abs(r["veff"]) < TOL_V
    assert rel(eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1], r["F"][:N - 1]) < TOL_F
    assert rel(eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1], r["Heta"][:N - 1]) < TOL_H
    assert rel(G, r["G"]) < TOL_F
    # the FD path (skip radius rc + 2h) against the oracle's analytic H eta, on the beads whose
    # eta does not span the 0.25 nm jump (there eps = h / max |eta| is 60 times smaller and FD's
    # own rounding error grows accordingly)
    ef = mop.Engine(w.system, hvp_mode=mop.MOP_HVP_FD, fd_h=1e-4)
    ef.set_path(0, X)
    ef.veff_and_grad(0)
    keep = [0, 1, 3, 4]
    assert rel(ef.get_field(0, mop.MOP_FIELD_HETA)[keep], r["Heta"][keep]) < 1e-3


@pytest.mark.slow
def test_cfg3_autograd_gradient_matches_central_differences():
    """Q = 24,000, N = 128: the gradient that the torch.autograd.Function returns, checked
    against central differences of V_eff on 64 seeded coordinates per bead for beads 1, 2, 64
    and N.  The differences are taken in FP64 by the oracle: moving coordinate k of bead n
    changes U (bead 1), the spring of eta^{n-1} through R^n alone, and the spring of eta^n through
    R^n and F^n(R^n), so V(+) - V(-) is summed from those terms only, atom by atom, with the
    perturbed bead's forces recomputed at both points (no cancellation between large sums)."""
    import torch
    w = workload(3)
    X = w.paths[0]
    N, Q = X.shape[0], X.shape[1]
    eng = mop.Engine(w.system)
    coords = torch.tensor(X, device="cuda", requires_grad=True)
    V = mop.veff(coords, eng, 0)
    V.backward()
    torch.cuda.synchronize()
    G = coords.grad.double().cpu().numpy()
    o = oracle.Oracle(w.system)
    s = w.system
    m = np.asarray(s.mass, np.float64)
    K = m * s.nu_path / (2.0 * s.dt_path)
    c = s.dt_path / (m * s.nu_path)
    Xd = X.astype(np.float64)
    h = 1e-5
    rng = np.random.default_rng(3003)
    beads = [0, 1, N // 2, N - 1]
    base_F = {}
    for n in beads:
        if n < N - 1:
            base_F[n] = o.forces(Xd[n])
    jobs = []
    for n in beads:
        for k in rng.choice(Q * 3, size=64, replace=False):
            jobs.append((n, int(k) // 3, int(k) % 3))

    def central(job):
        n, a, d = job
        dv = 0.0
        if n > 0:   # eta^{n-1} moves by +-h e in atom a only: K_a/2 (|e + h|^2 - |e - h|^2)
            e_prev = Xd[n][a, d] - Xd[n - 1][a, d] - c[a] * base_F_prev[n][a, d]
            dv += 2.0 * K[a] * h * e_prev
        if n < N - 1:
            xp, xm = Xd[n].copy(), Xd[n].copy()
            xp[a, d] += h
            xm[a, d] -= h
            Fp, Up = o.forces(xp)
            Fm, Um = o.forces(xm)
            ep = Xd[n + 1] - xp - c[:, None] * Fp
            em = Xd[n + 1] - xm - c[:, None] * Fm
            dv += float(np.sum(0.5 * K[:, None] * (ep - em) * (ep + em)))
            if n == 0:
                dv += Up - Um
        return dv / (2.0 * h)

    base_F_prev = {}
    for n in beads:
        if n > 0:
            base_F_prev[n] = base_F[n - 1][0] if (n - 1) in base_F else o.forces(Xd[n - 1])[0]
    with ThreadPoolExecutor(max_workers=max(1, oracle.num_threads())) as ex:
        fd = np.array(list(ex.map(central, jobs)))
    an = np.array([G[n, a, d] for n, a, d in jobs])
    e = float(np.linalg.norm(an - fd) / np.linalg.norm(fd))
    emax = float(np.max(np.abs(an - fd) / np.maximum(np.abs(fd), 1e-3 * np.sqrt(np.mean(fd ** 2)))))
    print(f"cfg3 autograd gradient vs FP64 central differences on {len(jobs)} coordinates: "
          f"relative 2-norm {e:.2e}, largest relative {emax:.2e}")
    assert e < TOL_F, e


@pytest.mark.parametrize("hvp_mode", [mop.MOP_HVP_ADJOINT, mop.MOP_HVP_FD])
def test_half_list_kernels_match_oracle(monkeypatch, hvp_mode):
    """The half-list pair kernels (MOP_PAIR_KERNELS=half, kept beside the bead-lane kernels for
    comparison) against the oracle on the water box: forces, H eta (the FD mode against the
    oracle's own Eq. 5 at the same h) and the gradient."""
    monkeypatch.setenv("MOP_PAIR_KERNELS", "half")
    w = workload(2, n_beads=16)
    X = w.paths[0]
    N = X.shape[0]
    kw = dict(hvp_mode=hvp_mode, fd_h=1e-3) if hvp_mode == mop.MOP_HVP_FD else {}
    eng, g = gpu_eval(w, **kw)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "Heta"),
                                     **(dict(hvp_mode=oracle.HVP_FD_EQ5, fd_h=1e-3) if kw else {}))
    errs = dict(F=rel(g["F"][:N - 1], r["F"][:N - 1]), Heta=rel(g["Heta"][:N - 1], r["Heta"][:N - 1]),
                G=rel(g["G"], r["G"]), V=abs(g["veff"] - r["veff"]) / abs(r["veff"]))
    print("half-list kernels", hvp_mode, errs)
    assert errs["F"] < TOL_F and errs["V"] < TOL_V
    assert errs["Heta"] < (1e-4 if kw else TOL_H) and errs["G"] < (1e-4 if kw else TOL_F)


@pytest.mark.parametrize("kernels", ["default", "blhalf", "blfull"])
@pytest.mark.parametrize("relaxed", [False, True])
@pytest.mark.parametrize("hvp_mode", [mop.MOP_HVP_ADJOINT, mop.MOP_HVP_FD])
def test_bead_lane_lists_match_oracle(monkeypatch, hvp_mode, relaxed, kernels):
    """The bead-lane kernels in their three arrangements against the oracle on the water box with
    70 beads (two bead groups, the second ragged): the default (full list; the H eta pass over the
    owner entries only, the j-atom's share added by 64-bit integer atomics to fixed-point sums, a
    self entry's pairs j > i), MOP_PAIR_KERNELS=blhalf (the half list in both passes) and =blfull
    (every entry in both passes, no atomics).  Forces, eta, H eta (FD: against the oracle's own
    Eq. 5 at the same h), the gradient, V_eff, and the per-row bars."""
    if kernels == "default":
        monkeypatch.delenv("MOP_PAIR_KERNELS", raising=False)
    else:
        monkeypatch.setenv("MOP_PAIR_KERNELS", kernels)
    w = workload(2, n_beads=70, relaxed=relaxed)
    X = w.paths[0]
    N = X.shape[0]
    fd = hvp_mode == mop.MOP_HVP_FD
    kw = dict(hvp_mode=hvp_mode, fd_h=1e-3) if fd else {}
    eng, g = gpu_eval(w, **kw)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"),
                                     **(dict(hvp_mode=oracle.HVP_FD_EQ5, fd_h=1e-3) if fd else {}))
    errs = dict(F=rel(g["F"][:N - 1], r["F"][:N - 1]), eta=rel(g["eta"][:N - 1], r["eta"][:N - 1]),
                Heta=rel(g["Heta"][:N - 1], r["Heta"][:N - 1]), G=rel(g["G"], r["G"]),
                V=abs(g["veff"] - r["veff"]) / abs(r["veff"]), U1=abs(g["U1"] - r["U1"]) / abs(r["U1"]))
    print("bead-lane", kernels, hvp_mode, relaxed, errs)
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["V"] < TOL_V and errs["U1"] < TOL_V
    assert_rows(g["F"][:N - 1], r["F"][:N - 1], TOL_F, "F")
    assert_rows(g["eta"][:N - 1], r["eta"][:N - 1], TOL_F, "eta")
    if fd:
        # FP32 central differences at h = 1e-3 nm: 30 times the rounding scale, as for the
        # full-list FD kernel
        assert errs["Heta"] < 1e-4 and errs["G"] < 1e-4
    else:
        assert errs["Heta"] < TOL_H and errs["G"] < TOL_F
        assert_rows(g["Heta"][:N - 1], r["Heta"][:N - 1], TOL_H, "Heta")
        assert_rows(g["G"], r["G"], TOL_F, "G")


@pytest.mark.parametrize("kernels", ["blhalf", "blfull"])
def test_bead_lane_lists_ewald_match_oracle(monkeypatch, kernels):
    """The bead-lane kernels on both lists with Ewald real space and SPME against the oracle."""
    from paper_2501_11962_b300 import synth
    monkeypatch.setenv("MOP_PAIR_KERNELS", kernels)
    w = workload(2, n_beads=6)
    sys = synth.with_pme(w.system)
    X = w.paths[0]
    N = X.shape[0]
    eng = mop.Engine(sys)
    eng.set_path(0, X)
    v, G = eng.veff_and_grad(0)
    r = oracle.Oracle(sys).veff_pme(X.astype(np.float64))
    F = eng.get_field(0, mop.MOP_FIELD_FORCE)[:N - 1]
    H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
    errs = dict(F=rel(F, r["F"][:N - 1]), Heta=rel(H, r["Heta"][:N - 1]), G=rel(G, r["G"]),
                V=abs(v[0] - r["veff"]) / abs(r["veff"]))
    print("bead-lane", kernels, "SPME", errs)
    assert errs["F"] < TOL_F and errs["G"] < TOL_F and errs["Heta"] < TOL_H and errs["V"] < TOL_V, errs


@pytest.mark.parametrize("kernels", ["default", "blhalf"])
@pytest.mark.parametrize("relaxed", [False, True])
@pytest.mark.parametrize("hvp_mode", [mop.MOP_HVP_ADJOINT, mop.MOP_HVP_FD])
def test_j_side_sums_are_bitwise_reproducible(monkeypatch, hvp_mode, relaxed, kernels):
    """The j-side sums (the H eta pass over the owner entries of the full list, by default, and
    both passes of the half list) are added by atomics in whatever order the warps run; they are
    64-bit fixed-point integers, so every addition is exact and two handles give the same bits
    (config 4's 96-bead path, around the generated structure with forces up to 2e5 kJ/mol/nm, and
    around the relaxed one)."""
    if kernels == "default":
        monkeypatch.delenv("MOP_PAIR_KERNELS", raising=False)
    else:
        monkeypatch.setenv("MOP_PAIR_KERNELS", kernels)
    w = workload(4, relaxed=relaxed)
    kw = dict(hvp_mode=hvp_mode, fd_h=1e-3) if hvp_mode == mop.MOP_HVP_FD else {}
    outs = []
    for _ in range(2):
        eng = mop.Engine(w.system, **kw)
        eng.set_path(0, w.paths[3])
        v, G = eng.veff_and_grad(0)
        outs.append((v[0], G, eng.get_field(0, mop.MOP_FIELD_FORCE), eng.get_field(0, mop.MOP_FIELD_HETA)))
        eng.close()
    for name, a, b in zip(("V", "G", "F", "Heta"), outs[0], outs[1]):
        d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
        assert np.array_equal(a, b), (name, int(np.count_nonzero(d)), float(np.abs(d).max()))


@pytest.mark.parametrize("relaxed", [False, True])
def test_cfg3_fields_match_oracle(relaxed):
    """Config 3 (Q = 24,000 waters, N = 128: two full bead groups, the second one bead short in
    the force and H eta passes): F, eta, H eta and G element by element and per row, V_eff."""
    w = workload(3, relaxed=relaxed)
    X = w.paths[0]
    N = X.shape[0]
    eng, g = gpu_eval(w)
    r = oracle.Oracle(w.system).veff(X.astype(np.float64), want=("G", "F", "eta", "Heta"))
    errs = dict(F=rel(g["F"][:N - 1], r["F"][:N - 1]), eta=rel(g["eta"][:N - 1], r["eta"][:N - 1]),
                Heta=rel(g["Heta"][:N - 1], r["Heta"][:N - 1]), G=rel(g["G"], r["G"]),
                V=abs(g["veff"] - r["veff"]) / abs(r["veff"]))
    print("cfg3", relaxed, errs)
    assert errs["F"] < TOL_F and errs["eta"] < TOL_F and errs["G"] < TOL_F
    assert errs["Heta"] < TOL_H and errs["V"] < TOL_V
    assert_rows(g["F"][:N - 1], r["F"][:N - 1], TOL_F, "cfg3 F")
    assert_rows(g["Heta"][:N - 1], r["Heta"][:N - 1], TOL_H, "cfg3 Heta")
    assert_rows(g["G"], r["G"], TOL_F, "cfg3 G")
