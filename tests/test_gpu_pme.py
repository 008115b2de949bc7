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
